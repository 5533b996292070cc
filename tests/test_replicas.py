"""Multi-rank control of the benchmark's replica mode on CPU (gloo, world size 2)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1008_2865_gb300 import replicas  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    replicas.init("gloo")
    ws, r, lr = replicas.world()
    replicas.barrier()
    # rank r processed (r + 1) * 1e6 units in (r + 1) seconds
    v = replicas.weak_scaling_value((r + 1) * 1e6, float(r + 1))
    out[rank] = (ws, r, lr, replicas.max_over_ranks(r * 10.0), replicas.sum_over_ranks(1.0),
                 replicas.seed_for_rank(7, r), v)
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    res = [out[r] for r in range(world)]
    for r, (ws, rank, lr, mx, sm, seed, v) in enumerate(res):
        assert (ws, rank, lr) == (2, r, r)
        assert mx == 10.0 and sm == 2.0
        assert seed == 7 + r
        # total 3e6 units, slowest rank 2 s -> 1.5 "mega-units" per second
        assert v == pytest.approx(1.5)
    assert res[0][5] != res[1][5]


def test_single_process_defaults():
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert replicas.world() == (1, 0, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.weak_scaling_value(2e6, 2.0) == pytest.approx(1.0)
