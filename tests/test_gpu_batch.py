"""GPU tests of the batched mode: uneven replicas advanced by one launch per step.

A replica in a batch must reproduce, bit for bit, the same lattice run alone
with the same tile shape (same per-tile code, same reduction order), with and
without CUDA-graph replay; one replica is also compared with the oracle."""
import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import Batch, LBError, Lattice, capi, inputs

pytestmark = pytest.mark.gpu

SHAPES = [(64, 48), (131, 67), (192, 192), (300, 40), (5, 5)]
G2S = [0.0, 0.3, 0.6, 0.9, 0.45]


def _rhos():
    return [inputs.noisy_density(nx, ny, seed=1000 + i, mean=0.7, amp=0.01, mode="rel")
            for i, (nx, ny) in enumerate(SHAPES)]


@pytest.mark.parametrize("use_graph,launch", [(1, (128, 32)), (0, (128, 32)), (1, (64, 16)),
                                              (1, (256, 48))])
def test_batch_matches_single_runs_bit_for_bit(use_graph, launch):
    rhos = _rhos()
    steps = 37            # crosses graph periods and a ragged tail of direct launches
    with Batch(rhos, G1=-5.0, G2=G2S, trace_every=10) as b:
        b.set_launch(launch[0], launch[1], use_graph)
        b.step(steps)
        assert b.t == steps and len(b) == len(rhos)
        assert capi.lb_batch_check_guards(b.handle) == 0
        got = [(b.fields(i), b.trace(i), b.energy(i)) for i in range(len(rhos))]
    for i, r in enumerate(rhos):
        with Lattice(r, G1=-5.0, G2=G2S[i], trace_every=10) as lat:
            lat.set_launch(launch[0], launch[1], 0)
            lat.step(steps)
            f = lat.fields()
            tr = lat.trace()
            en = lat.energy()
        for a, c in zip(got[i][0], f):
            assert np.array_equal(a, c)
        assert np.array_equal(got[i][1], tr)
        assert got[i][2] == en


@pytest.mark.parametrize("launch,prec", [((128, 72), "fp32"), ((128, 16), "fp32"), ((64, 8), "fp32"),
                                         ((128, 72), "fp16_delta")])
def test_batch_replicas_march_as_they_do_alone(launch, prec):
    """A lattice whose state exceeds L2 (1536^2 x 80 B = 189 MB) marches down in even row
    chunks and up in odd ones, in plain and reduction steps; in a batch it marches the
    same way, next to a small replica (96 x 80) that marches down, so both replicas'
    fields and traces are bit-identical to their single runs. (That the direction does
    not change the fields is checked against the oracle by the sampled 8192^2 and
    15424^2 tests, whose steps alternate.)"""
    n = 1536
    rhos = [inputs.noisy_density(n, n, seed=77, mean=0.7, amp=0.01, mode="rel"),
            inputs.noisy_density(96, 80, seed=78, mean=0.7, amp=0.01, mode="rel")]
    steps = 23
    alone = []
    for r in rhos:
        with Lattice(r, G1=-5.0, G2=0.6, trace_every=10, prec=prec) as lat:
            lat.set_launch(launch[0], launch[1], 0)
            lat.step(steps)
            alone.append((lat.fields(), lat.trace()))
    with Batch(rhos, G1=-5.0, G2=[0.6, 0.6], trace_every=10, prec=prec) as b:
        b.set_launch(launch[0], launch[1], 1)
        b.step(steps)
        batched = [(b.fields(i), b.trace(i)) for i in range(2)]
    for (f1, t1), (f2, t2) in zip(alone, batched):
        for a, c in zip(f1, f2):
            assert np.array_equal(a, c)
        assert len(t1) == 3 and np.array_equal(t1, t2)
    assert alone[0][0][0].max() - alone[0][0][0].min() > 0.01       # the flow has structure
    if prec == "fp32":
        # the alternating reduction step at t = 0 against the oracle's Sec. 5 sums of the
        # initial state, within the bound of the FP32 per-thread partials (63 u)
        tr = alone[0][1]
        ref = oracle.energy(oracle.psi(rhos[0]), -5.0, 0.6)
        for got, want in zip(tr[0, 2:5], ref):
            assert abs(got - want) <= 4e-6 * abs(want)
        assert abs(tr[0, 1] - rhos[0].sum()) <= 1e-6 * rhos[0].sum()


def test_batch_replica_matches_oracle_and_omega():
    rhos = [inputs.noisy_density(96, 80, seed=5, amp=0.01, mode="rel"),
            inputs.noisy_density(128, 64, seed=6, amp=0.01, mode="rel")]
    with Batch(rhos, omega=[1.0, 1.3], G1=-5.0, G2=[0.6, 0.2], trace_every=10) as b:
        b.step(100)
        res = [b.fields(i) for i in range(2)]
        trs = [b.trace(i) for i in range(2)]
    for i, (om, g2) in enumerate([(1.0, 0.6), (1.3, 0.2)]):
        ref = oracle.run(rhos[i], 100, omega=om, G1=-5.0, G2=g2, trace_every=10)
        rho, ux, uy = res[i]
        assert np.max(np.abs(rho - ref[0])) / np.max(ref[0]) <= 1e-5
        assert np.max(np.abs(ux - ref[1])) / np.max(np.abs(ref[1])) <= 1e-5
        assert np.array_equal(trs[i][:, 0], ref[3][:, 0])
        assert np.max(np.abs(trs[i][:, 1:] - ref[3][:, 1:]) / np.abs(ref[3][:, 1:])) <= 1e-4


def test_batch_arguments():
    rhos = _rhos()[:2]
    with pytest.raises(LBError):
        capi.lb_batch_init([capi.make_params(64, 48, prec="fp64"),
                            capi.make_params(131, 67, prec="fp64")], rhos)
    with pytest.raises(LBError):
        capi.lb_batch_init([capi.make_params(64, 48, trace_every=10),
                            capi.make_params(131, 67, trace_every=5)], rhos)
    with Batch(rhos) as b:
        with pytest.raises(LBError):
            b.energy(2)
        with pytest.raises(LBError):
            b.set_launch(100, 32)
        assert b.launch == (128, 32, 1)
