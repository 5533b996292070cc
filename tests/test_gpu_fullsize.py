"""GPU parity at the workloads' own sizes and launch shapes.

- The 1024^2 G2 sweep's lattices (G2 in {0, 0.3, 0.6, 0.9}, rho = 0.7 (1 +- 1%),
  the sweep's seeds 2..5), 100 steps, every site against the FP64 oracle.
- A 2048^2 lattice (state 335 MB, larger than L2, so plain and reduction steps
  march in alternating directions) in the 8192^2 benchmark's launch shape,
  100 steps, every site and the ten trace rows against the oracle.
- FP16 storage at 8192^2 in the FP16 benchmark's launch shape, 3 steps, sampled
  sites against oracle patches (dependency cone of radius 9).
- The 96-replica sweep (32 each of 192^2, 384^2, 640^2) in the benchmark's batch
  launch: one replica of each size bit-identical to its single run, fields and
  trace, and the 192^2 replica against the oracle.

Bars as in test_gpu_parity: FP32 1e-5 (max |d| over max |reference|), mass 1e-6,
trace 1e-4; FP16 storage the bars of test_fp16_delta_storage_error_bound.
"""
import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import Batch, Lattice, inputs

pytestmark = pytest.mark.gpu


def _norm_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _trace_err(tr, ref):
    worst = 0.0
    for c in range(1, 5):
        r = ref[:, c]
        if np.all(r == 0):
            worst = max(worst, float(np.max(np.abs(tr[:, c]))))
        else:
            worst = max(worst, float(np.max(np.abs(tr[:, c] - r) / np.abs(r))))
    return worst


def _gpu_run(rho0, steps, launch=None, **kw):
    with Lattice(rho0, **kw) as lat:
        if launch:
            lat.set_launch(*launch)
        lat.step(steps)
        return lat.fields() + (lat.trace(),)


@pytest.mark.parametrize("i,G2", list(enumerate((0.0, 0.3, 0.6, 0.9))))
def test_sweep_1024_lattices_100_steps(i, G2):
    rho0 = inputs.noisy_density(1024, 1024, 2 + i, mean=0.7, amp=0.01, mode="rel")
    ref = oracle.run(rho0, 100, G1=-5.0, G2=G2, trace_every=10)
    rho, ux, uy, tr = _gpu_run(rho0, 100, G1=-5.0, G2=G2, trace_every=10)
    assert _norm_err(rho, ref[0]) <= 1e-5
    assert _norm_err(ux, ref[1]) <= 1e-5 and _norm_err(uy, ref[2]) <= 1e-5
    assert np.array_equal(tr[:, 0], ref[3][:, 0])
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-6
    assert _trace_err(tr, ref[3]) <= 1e-4


def test_alternating_march_2048_bench_shape_100_steps():
    n = 2048
    assert n * n * 80 > 128 * 2 ** 20          # the steps alternate their march
    rho0 = inputs.noisy_density(n, n, 21, mean=0.7, amp=0.01, mode="rel")
    ref = oracle.run(rho0, 100, G1=-5.0, G2=0.6, trace_every=10)
    rho, ux, uy, tr = _gpu_run(rho0, 100, launch=(128, 72, 0), G1=-5.0, G2=0.6, trace_every=10)
    assert _norm_err(rho, ref[0]) <= 1e-5
    assert _norm_err(ux, ref[1]) <= 1e-5 and _norm_err(uy, ref[2]) <= 1e-5
    assert len(tr) == 10 and np.array_equal(tr[:, 0], ref[3][:, 0])
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-6
    assert _trace_err(tr, ref[3]) <= 1e-4


def test_fp16_storage_full_size_8192_sampled():
    torch = pytest.importorskip("torch")
    from paper_1008_2865_gb300 import tune
    n, steps, R = 8192, 3, 9
    rho0 = inputs.noisy_density(n, n, seed=7, mean=0.7, amp=0.01, mode="rel")
    launch = tune.lookup(n, n, "fp16_delta") or (64, 72, 0)
    rng = np.random.default_rng(15)
    ys = np.array(list(rng.integers(0, n, 20)) + [0, n - 1, n - 1, 71, 72])
    xs = np.array(list(rng.integers(0, n, 20)) + [n - 1, 0, n - 1, 61, 62])
    with Lattice(torch.from_numpy(rho0).cuda(), prec="fp16_delta", G1=-5.0, G2=0.6,
                 trace_every=10) as lat:
        lat.set_launch(*launch)
        lat.step(steps)
        f = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
        lat.fields(f[0], f[1], f[2])
        iy, ix = torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()
        got = f[:, iy, ix].cpu().numpy()
        umax = float(f[1:].abs().max())
        del f
    worst = [0.0, 0.0]
    for k, (y, x) in enumerate(zip(ys, xs)):
        patch = rho0[np.ix_(np.arange(y - R, y + R + 1) % n, np.arange(x - R, x + R + 1) % n)]
        r, ux, uy, _ = oracle.run(patch, steps, G1=-5.0, G2=0.6)
        worst[0] = max(worst[0], abs(got[0, k] - r[R, R]))
        worst[1] = max(worst[1], abs(got[1, k] - ux[R, R]), abs(got[2, k] - uy[R, R]))
    assert worst[0] <= 1e-4 * 0.71
    assert worst[1] <= 1e-2 * umax


def test_batch_sweep_96_replicas_match_single_runs():
    from paper_1008_2865_gb300 import tune
    sizes = [s for s in (192, 384, 640) for _ in range(32)]
    g2 = inputs.g2_sweep(len(sizes), seed=100)
    rhos = [inputs.noisy_density(s, s, 1000 + i, mean=0.7, amp=0.01, mode="rel")
            for i, s in enumerate(sizes)]
    shape = tune.lookup_batch([r.shape for r in rhos]) or (64, 32)
    steps = 25                                  # crosses three reduction steps
    picks = (0, 32, 64)                         # one replica of each size
    with Batch(rhos, G1=-5.0, G2=list(g2), trace_every=10) as b:
        b.set_launch(shape[0], shape[1], 1)
        b.step(steps)
        got = {i: (b.fields(i), b.trace(i)) for i in picks}
    for i in picks:
        with Lattice(rhos[i], G1=-5.0, G2=float(g2[i]), trace_every=10) as lat:
            lat.set_launch(shape[0], shape[1], 0)
            lat.step(steps)
            fields, tr = lat.fields(), lat.trace()
        for a, c in zip(got[i][0], fields):
            assert np.array_equal(a, c)
        assert len(tr) == 3 and np.array_equal(got[i][1], tr)
    ref = oracle.run(rhos[0], steps, G1=-5.0, G2=float(g2[0]), trace_every=10)
    rho, ux, uy = got[0][0]
    assert _norm_err(rho, ref[0]) <= 1e-5
    assert _norm_err(ux, ref[1]) <= 1e-5 and _norm_err(uy, ref[2]) <= 1e-5
    assert _trace_err(got[0][1], ref[3]) <= 1e-4
