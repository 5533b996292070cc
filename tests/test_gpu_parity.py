"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (written here, from the targets the method is held to):
  FP64 mode:  <= 1e-12 relative in rho and u over 1000 steps (the FP64 path
              follows the oracle's operation order, so it is expected exact);
  FP32 mode:  <= 1e-5 over 100 steps, measured as max|d rho| / max|rho| and
              max|d u| / max|u| (u starts at 0, so pointwise relative error is
              ill-posed); mass to 1e-6; pseudo-energy trace to 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import LBError, Lattice, capi, inputs

pytestmark = pytest.mark.gpu


def _norm_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _trace_err(tr, ref):
    """Largest relative deviation of energy/mass columns; a column that is exactly
    zero in the reference (E_m when G2 = 0) must be zero here too."""
    worst = 0.0
    for c in range(1, 5):
        r = ref[:, c]
        if np.all(r == 0):
            worst = max(worst, float(np.max(np.abs(tr[:, c]))))
        else:
            worst = max(worst, float(np.max(np.abs(tr[:, c] - r) / np.abs(r))))
    return worst


def _run_gpu(rho0, steps, prec="fp32", launch=None, **kw):
    with Lattice(rho0, prec=prec, **kw) as lat:
        if launch:
            lat.set_launch(*launch)
        lat.step(steps)
        rho, ux, uy = lat.fields()
        tr = lat.trace()
        en = lat.energy()
        assert lat.t == steps
        # no kernel wrote outside any of the state's buffers
        assert capi.lb_check_guards(lat.handle) == 0
    return rho, ux, uy, tr, en


# ----------------------------------------------------------------- FP64 parity
@pytest.mark.parametrize("G2", [0.0, 0.5])
def test_fp64_1000_steps_128(G2):
    """128x128, omega = 1, G1 = -5, rho = 0.7 + U(-0.01, 0.01), 1000 steps, trace every 10."""
    rho0 = inputs.noisy_density(128, 128, seed=1, mean=0.7, amp=0.01, mode="abs")
    ref = oracle.run(rho0, 1000, G1=-5.0, G2=G2, trace_every=10)
    rho, ux, uy, tr, en = _run_gpu(rho0, 1000, prec="fp64", G1=-5.0, G2=G2, trace_every=10)
    assert _norm_err(rho, ref[0]) <= 1e-12
    assert _norm_err(ux, ref[1]) <= 1e-12 and _norm_err(uy, ref[2]) <= 1e-12
    assert tr.shape == ref[3].shape == (100, 5)
    assert np.array_equal(tr[:, 0], ref[3][:, 0])
    assert _trace_err(tr, ref[3]) <= 1e-12
    # phase separation happened: this is not a near-uniform comparison
    assert rho.max() > 1.5 and rho.min() < 0.3


def test_fp64_is_bit_exact_over_short_runs():
    """Same operation order and a correctly rounded exp: identical bits."""
    rho0 = inputs.noisy_density(37, 29, seed=2, mean=0.7, amp=0.05)
    for G2, omega in [(0.0, 1.0), (0.7, 1.3)]:
        ref = oracle.run(rho0, 25, omega=omega, G1=-5.0, G2=G2)
        rho, ux, uy, _, _ = _run_gpu(rho0, 25, prec="fp64", omega=omega, G1=-5.0, G2=G2)
        assert np.array_equal(rho, ref[0]) and np.array_equal(ux, ref[1])
        assert np.array_equal(uy, ref[2])


# ----------------------------------------------------------------- FP32 parity
FP32_CASES = [
    # (nx, ny, G2, omega, noise mode, seed, steps)
    (128, 128, 0.0, 1.0, "abs", 1, 100),
    (128, 128, 0.5, 1.0, "abs", 1, 100),
    (300, 200, 0.6, 1.0, "rel", 2, 100),     # 3 ragged strips, ragged last row chunk
    (131, 67, 0.9, 1.0, "rel", 3, 100),
    (256, 256, 0.3, 1.3, "rel", 4, 100),     # omega != 1 exercises (1 - omega) f
    (1024, 40, 0.6, 1.0, "rel", 8, 100),     # many strips, one short chunk
    # Lattices too small for any unstable mode: the noise decays and u -> 0
    # (1e-17 after 100 steps), so max|u| cannot normalise the error there; they
    # are compared while the flow is still O(1e-4).
    (5, 5, 0.5, 1.0, "abs", 5, 10),          # smallest lattice the stencil allows
    (6, 7, 0.0, 0.9, "abs", 6, 10),
    (5, 9, 0.6, 1.0, "abs", 7, 10),
]


@pytest.mark.parametrize("nx,ny,G2,omega,mode,seed,steps", FP32_CASES)
def test_fp32_parity(nx, ny, G2, omega, mode, seed, steps):
    rho0 = inputs.noisy_density(nx, ny, seed=seed, mean=0.7, amp=0.01, mode=mode)
    ref = oracle.run(rho0, steps, omega=omega, G1=-5.0, G2=G2, trace_every=10)
    rho, ux, uy, tr, en = _run_gpu(rho0, steps, omega=omega, G1=-5.0, G2=G2, trace_every=10)
    assert _norm_err(rho, ref[0]) <= 1e-5
    assert _norm_err(ux, ref[1]) <= 1e-5 and _norm_err(uy, ref[2]) <= 1e-5
    assert np.array_equal(tr[:, 0], ref[3][:, 0])
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-6          # mass
    assert _trace_err(tr, ref[3]) <= 1e-4


@pytest.mark.parametrize("nx,launch", [(301, (64, 16, 0)), (301, (96, 17, 0)), (301, (128, 16, 0)),
                                       (301, (192, 40, 0)), (301, (256, 33, 0)),
                                       (320, (64, 16, 1)), (320, (128, 23, 1)),
                                       (320, (256, 40, 1)), (512, (128, 64, 1))])
def test_fp32_launch_shapes_agree(nx, launch):
    """Every CTA shape and both pipelines give the trajectory of the oracle (tile edges,
    halo columns, ragged strips and row chunks, periodic wrap of the copy windows)."""
    rho0 = inputs.noisy_density(nx, 170, seed=9, mean=0.7, amp=0.01, mode="rel")
    ref = oracle.run(rho0, 60, G1=-5.0, G2=0.6, trace_every=10)
    rho, ux, uy, tr, _ = _run_gpu(rho0, 60, launch=launch, G1=-5.0, G2=0.6, trace_every=10)
    assert _norm_err(rho, ref[0]) <= 1e-5
    assert _norm_err(ux, ref[1]) <= 1e-5 and _norm_err(uy, ref[2]) <= 1e-5
    assert _trace_err(tr, ref[3]) <= 1e-4


def test_fp32_energy_entry_matches_oracle_energy():
    rho0 = inputs.noisy_density(90, 77, seed=10, mean=0.7, amp=0.01, mode="rel")
    with Lattice(rho0, G1=-5.0, G2=0.6) as lat:
        lat.step(40)
        es, em, eb, mass = lat.energy()
        rho, _, _ = lat.fields()
    ref = oracle.run(rho0, 40, G1=-5.0, G2=0.6)
    ps = oracle.psi(ref[0])
    res, rem, reb = oracle.energy(ps, -5.0, 0.6)
    assert abs(es - res) <= 1e-4 * abs(res) and abs(em - rem) <= 1e-4 * abs(rem)
    assert abs(eb - reb) <= 1e-4 * abs(reb)
    assert abs(mass - rho0.sum()) <= 1e-6 * rho0.sum()


def test_fp32_is_deterministic():
    rho0 = inputs.noisy_density(200, 150, seed=11, mean=0.7, amp=0.01, mode="rel")
    a = _run_gpu(rho0, 50, G1=-5.0, G2=0.6, trace_every=5)
    b = _run_gpu(rho0, 50, G1=-5.0, G2=0.6, trace_every=5)
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)


# ----------------------------------------------------------------- long-run observables
def test_fp32_flat_interface_coexistence_densities():
    """Coexistence densities of a flat interface agree with the oracle to 1e-3."""
    nx, ny = 64, 5
    x = np.arange(nx) + 0.5
    prof = 0.156 + (1.93 - 0.156) * 0.5 * (np.tanh((x - 16) / 3) - np.tanh((x - 48) / 3))
    rho0 = prof[None, :].repeat(ny, 0)
    ref = oracle.run(rho0, 20000, G1=-5.0, G2=0.0)
    rho, _, _, _, _ = _run_gpu(rho0, 20000, G1=-5.0, G2=0.0, trace_every=0)
    for xs in (0, 32):
        assert abs(rho[2, xs] - ref[0][2, xs]) <= 1e-3 * ref[0][2, xs]


def test_fp32_mass_and_energy_trace_2000_steps():
    rho0 = inputs.noisy_density(256, 256, seed=12, mean=0.7, amp=0.01, mode="rel")
    ref = oracle.run(rho0, 2000, G1=-5.0, G2=0.6, trace_every=10)
    rho, ux, uy, tr, _ = _run_gpu(rho0, 2000, G1=-5.0, G2=0.6, trace_every=10)
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-6
    # the trace stays within 1e-4 while the two trajectories are still close
    early = tr[:, 0] <= 300
    assert np.max(np.abs(tr[early, 2:] - ref[3][early, 2:]) / np.abs(ref[3][early, 2:])) <= 1e-4


# ----------------------------------------------------------------- full size, sampled
def test_fp32_full_size_8192_sampled():
    """The 8192^2 roofline workload in the bench's launch shape, 3 steps: sampled sites
    against the oracle run on a periodic 19x19 patch around each site (the dependency
    cone of 3 steps has radius 9, so the patch reproduces the full lattice there)."""
    torch = pytest.importorskip("torch")
    n, steps, R = 8192, 3, 9
    rho0 = inputs.noisy_density(n, n, seed=7, mean=0.7, amp=0.01, mode="rel")
    dev_rho = torch.from_numpy(rho0).cuda()
    with Lattice(dev_rho, G1=-5.0, G2=0.6, trace_every=10) as lat:
        lat.step(steps)
        out = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
        lat.fields(out[0], out[1], out[2])
        e = lat.energy()
    fields = out.cpu().numpy()
    del out, dev_rho
    rng = np.random.default_rng(5)
    ys = list(rng.integers(0, n, 40)) + [0, n - 1, 0, n - 1, 63, 64, 4095]
    xs = list(rng.integers(0, n, 40)) + [0, n - 1, n - 1, 0, 125, 126, 127]
    worst = [0.0, 0.0]
    for y, x in zip(ys, xs):
        yy = (np.arange(y - R, y + R + 1)) % n
        xx = (np.arange(x - R, x + R + 1)) % n
        patch = rho0[np.ix_(yy, xx)]
        r, ux, uy, _ = oracle.run(patch, steps, G1=-5.0, G2=0.6)
        worst[0] = max(worst[0], abs(fields[0, y, x] - r[R, R]))
        worst[1] = max(worst[1], abs(fields[1, y, x] - ux[R, R]), abs(fields[2, y, x] - uy[R, R]))
    assert worst[0] <= 1e-5 * 0.71
    assert worst[1] <= 1e-5 * max(np.max(np.abs(fields[1])), 1e-12)
    assert abs(e[3] - rho0.sum()) <= 1e-6 * rho0.sum()


def test_fp32_largest_square_lattice_sampled():
    """15424^2, the largest square lattice whose tiled populations (288 ceil(nx/32) ny
    elements) keep the 32-bit offsets of the step below 2^31 (15456^2 is rejected on the
    host). Three steps; sites near the last rows, the last tile column and the periodic
    edges against oracle patches, as in the 8192^2 test; mass exact to 1e-6."""
    torch = pytest.importorskip("torch")
    n, steps, R = 15424, 3, 9
    assert 288 * (n // 32) * n < 2 ** 31 <= 288 * ((n + 32) // 32) * (n + 32)
    rho0 = inputs.noisy_density(n, n, seed=8, mean=0.7, amp=0.01, mode="rel")
    rng = np.random.default_rng(6)
    ys = np.array(list(rng.integers(0, n, 12)) + [0, n - 1, n - 1, n - 2, 7711])
    xs = np.array(list(rng.integers(0, n, 12)) + [n - 1, 0, n - 1, n - 33, 7712])
    with Lattice(torch.from_numpy(rho0).cuda(), G1=-5.0, G2=0.6, trace_every=10) as lat:
        lat.step(steps)
        f = torch.empty((3, n, n), dtype=torch.float64, device="cuda")
        lat.fields(f[0], f[1], f[2])
        e = lat.energy()
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
    assert worst[0] <= 1e-5 * 0.71
    assert worst[1] <= 1e-5 * max(umax, 1e-12)
    assert abs(e[3] - rho0.sum()) <= 1e-6 * rho0.sum()


# ----------------------------------------------------------------- edge cases
def test_invalid_density_rejected():
    for bad in (np.nan, 0.0, -0.1, np.inf):
        rho0 = np.full((8, 8), 0.7)
        rho0[3, 4] = bad
        with pytest.raises(LBError) as ei:
            Lattice(rho0)
        assert ei.value.status == capi.LB_ERR_ARG


def test_step_arguments_and_time():
    rho0 = inputs.noisy_density(16, 16, seed=1)
    with Lattice(rho0) as lat:
        assert lat.t == 0
        lat.step(0)
        assert lat.t == 0
        with pytest.raises(LBError):
            capi.lb_step(lat.handle, -1)
        lat.step(7)
        assert lat.t == 7
        with pytest.raises(LBError):
            lat.set_launch(100, 16, 0)
        with pytest.raises(LBError):
            lat.set_launch(128, 3, 0)
        with pytest.raises(LBError):
            lat.set_launch(128, 16, 1)      # nx = 16 is too narrow for the copy windows
        with pytest.raises(LBError):
            lat.set_launch(128, 16, 2)


def test_device_pointers_and_partial_fields():
    torch = pytest.importorskip("torch")
    rho0 = inputs.noisy_density(40, 30, seed=3)
    with Lattice(torch.from_numpy(rho0).cuda(), G2=0.5) as lat:
        lat.step(20)
        r = torch.empty((30, 40), dtype=torch.float64, device="cuda")
        lat.fields(rho=r)
        h_rho, h_ux, _ = lat.fields()
        assert np.array_equal(r.cpu().numpy(), h_rho)
        only_ux = np.empty((30, 40))
        lat.fields(ux=only_ux)
        assert np.array_equal(only_ux, h_ux)


def test_pinned_host_buffers_match_pageable_and_device():
    """Pinned host memory is read (init) and written (fields) in place by the kernels;
    the results equal those through pageable host memory and device memory."""
    torch = pytest.importorskip("torch")
    rho0 = inputs.noisy_density(301, 77, seed=4, mean=0.7, amp=0.01, mode="rel")
    pinned_in = torch.from_numpy(rho0).pin_memory()
    res = []
    for src in (rho0, pinned_in, torch.from_numpy(rho0).cuda()):
        with Lattice(src, G1=-5.0, G2=0.6) as lat:
            lat.step(25)
            pageable = lat.fields()
            pinned = [torch.empty((77, 301), dtype=torch.float64).pin_memory() for _ in range(3)]
            lat.fields(*pinned)
            only_uy = torch.empty((77, 301), dtype=torch.float64).pin_memory()
            lat.fields(uy=only_uy)
            dev = [torch.empty((77, 301), dtype=torch.float64, device="cuda") for _ in range(3)]
            lat.fields(dev[0], dev[1], dev[2])
        for a, b, c in zip(pageable, pinned, dev):
            assert np.array_equal(a, b.numpy()) and np.array_equal(a, c.cpu().numpy())
        assert np.array_equal(pageable[2], only_uy.numpy())
        res.append(pageable)
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)


def test_guard_check_sees_a_write_outside_a_buffer():
    """The guard check is not vacuous: a byte changed just past a buffer (by a host-side
    cudaMemset through the test hook, never by a kernel) is reported, buffer by buffer."""
    with Lattice(inputs.noisy_density(40, 30, seed=1)) as lat:
        lat.step(3)
        assert capi.lb_check_guards(lat.handle) == 0
        capi.lb_debug_damage_guard(lat.handle, 0)
        assert capi.lb_check_guards(lat.handle) == 1
        capi.lb_debug_damage_guard(lat.handle, 3)
        assert capi.lb_check_guards(lat.handle) == 2
        with pytest.raises(LBError):
            capi.lb_debug_damage_guard(lat.handle, 10_000)


def test_pipeline_availability():
    with Lattice(inputs.noisy_density(512, 64, seed=1)) as lat:
        assert lat.launch[2] == 0                  # default: register prefetch
        lat.set_launch(128, 32, 1)                 # aligned and wide: rings allowed
        assert lat.launch == (128, 32, 1)
    with Lattice(inputs.noisy_density(301, 64, seed=1)) as lat:
        with pytest.raises(LBError):
            lat.set_launch(128, 32, 1)             # not a whole number of 32-column tiles
    with Lattice(inputs.noisy_density(516, 64, seed=1), prec="fp16_delta") as lat:
        with pytest.raises(LBError):
            lat.set_launch(128, 32, 1)             # 516 = 16 tiles + 4 columns


def test_bounded_wait_reports_timeout_and_context_survives():
    """Every CTA arms the barrier of its first row unit and issues none of that unit's
    copies (test hook), so that wait runs out with nothing of the unit in flight; the
    kernel returns, the next synchronising call reports LB_ERR_TIMEOUT, and the CUDA
    context keeps working for a fresh state."""
    rho0 = inputs.noisy_density(256, 48, seed=2)
    lat = Lattice(rho0, trace_every=0)
    lat.set_launch(128, 16, 1)
    with pytest.raises(LBError):
        capi.lb_set_wait_limit(lat.handle, 2_000_000, 2)  # the hook takes 0 or 1
    capi.lb_set_wait_limit(lat.handle, 2_000_000, 1)     # ~1 ms per wait
    lat.step(1)
    with pytest.raises(LBError) as ei:
        lat.energy()
    assert ei.value.status == capi.LB_ERR_TIMEOUT
    with pytest.raises(LBError) as ei:
        lat.step(1)
    assert ei.value.status == capi.LB_ERR_STATE
    lat.close()
    ref = oracle.run(rho0, 20, G1=-5.0, G2=0.0)
    rho, _, _, _, _ = _run_gpu(rho0, 20, G1=-5.0, G2=0.0, trace_every=0)
    assert _norm_err(rho, ref[0]) <= 1e-5


def test_trace_rows_and_ring():
    rho0 = inputs.noisy_density(24, 24, seed=4)
    with Lattice(rho0, trace_every=3) as lat:
        lat.step(10)
        tr = lat.trace()
        assert list(tr[:, 0]) == [0, 3, 6, 9]
        assert len(lat.trace(cap=2)) == 2 and list(lat.trace(cap=2)[:, 0]) == [6, 9]
    with Lattice(rho0, trace_every=0) as lat:
        lat.step(10)
        assert len(lat.trace()) == 0


def test_fp64_energy_matches_oracle():
    rho0 = inputs.noisy_density(33, 35, seed=6, amp=0.05)
    with Lattice(rho0, prec="fp64", G2=0.8) as lat:
        lat.step(30)
        es, em, eb, mass = lat.energy()
    ref = oracle.run(rho0, 30, G1=-5.0, G2=0.8)
    r = oracle.energy(oracle.psi(ref[0]), -5.0, 0.8)
    assert np.allclose([es, em, eb], r, rtol=1e-13, atol=0)
    assert abs(mass - ref[0].sum()) <= 1e-13 * mass


# ----------------------------------------------------------------- FP16 storage, droplets
@pytest.mark.parametrize("nx,mode,G2,rho_bar,u_bar", [(128, "abs", 0.0, 1e-3, 1e-2),
                                                      (256, "rel", 0.6, 1e-4, 1e-2)])
def test_fp16_delta_storage_error_bound(nx, mode, G2, rho_bar, u_bar):
    """Deviations stored in IEEE half (FP32 arithmetic): the error against FP64 after
    100 steps stays under the stated bound (measured 6.8e-4 / 3.1e-3 and 3.8e-5 / 4.7e-3)."""
    rho0 = inputs.noisy_density(nx, nx, seed=1, mean=0.7, amp=0.01, mode=mode)
    ref = oracle.run(rho0, 100, G1=-5.0, G2=G2, trace_every=10)
    rho, ux, uy, tr, _ = _run_gpu(rho0, 100, prec="fp16_delta", G1=-5.0, G2=G2, trace_every=10)
    assert _norm_err(rho, ref[0]) <= rho_bar
    assert max(_norm_err(ux, ref[1]), _norm_err(uy, ref[2])) <= u_bar
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-5


@pytest.mark.parametrize("G2", [0.0, 0.5])
def test_droplet_count_exact_fp64(G2):
    """Same trajectory, same droplets: the FP64 path's fields are the oracle's bit for
    bit, so the droplet count and perimeter agree exactly after phase separation."""
    from paper_1008_2865_gb300 import diag
    rho0 = inputs.noisy_density(128, 128, seed=1, mean=0.7, amp=0.01, mode="abs")
    ref = oracle.run(rho0, 1500, G1=-5.0, G2=G2)
    rho, _, _, _, _ = _run_gpu(rho0, 1500, prec="fp64", G1=-5.0, G2=G2, trace_every=0)
    n_gpu, _ = diag.droplets(rho)
    n_ref, _ = diag.droplets(ref[0])
    assert n_gpu == n_ref and n_ref >= 1
    assert diag.perimeter(rho) == diag.perimeter(ref[0])


def test_fp32_droplet_count_reproducible():
    from paper_1008_2865_gb300 import diag
    rho0 = inputs.noisy_density(256, 256, seed=3, mean=0.7, amp=0.01, mode="rel")
    counts = []
    for _ in range(2):
        rho, _, _, _, _ = _run_gpu(rho0, 1500, G1=-5.0, G2=0.6, trace_every=0)
        counts.append((diag.droplets(rho)[0], diag.perimeter(rho)))
    assert counts[0] == counts[1]


# ----------------------------------------------------------------- checkpoint / resume, blow-up
@pytest.mark.parametrize("prec", ["fp32", "fp64", "fp16_delta"])
def test_save_and_resume_is_bit_exact(prec):
    torch = pytest.importorskip("torch")
    rho0 = inputs.noisy_density(72, 40, seed=13, mean=0.7, amp=0.01, mode="rel")
    with Lattice(rho0, prec=prec, G2=0.6, trace_every=7) as a:
        a.step(30)
        saved = a.save()
        a.step(40)
        ref = a.fields()
        tr_ref = a.trace()
    # into a fresh state of the same shape (other initial density, same rho_ref)
    with Lattice(rho0[::-1].copy(), prec=prec, G2=0.6, trace_every=7,
                 rho_ref=float(np.float32(rho0.mean()))) as b:
        b.load(saved)
        assert b.t == 30
        b.step(40)
        got = b.fields()
        tr = b.trace()
    for u, v in zip(got, ref):
        assert np.array_equal(u, v)
    # the rows after the resume point agree bit for bit
    assert np.array_equal(tr[tr[:, 0] >= 30], tr_ref[tr_ref[:, 0] >= 30])
    # device buffers work too, and a mismatching header is refused
    with Lattice(rho0, prec=prec, G2=0.6, trace_every=0) as c:
        dev = torch.empty(capi.lb_state_bytes(c.handle), dtype=torch.uint8, device="cuda")
        c.save(dev)
        c.load(dev)
    with Lattice(inputs.noisy_density(40, 72, seed=1), prec=prec) as d:
        with pytest.raises(LBError):
            d.load(saved)


def test_blow_up_is_reported_as_nonfinite():
    """An absurd coupling drives the lattice to NaN; the fused reduction flags it and the
    next synchronising call reports LB_ERR_NONFINITE instead of returning garbage silently."""
    rho0 = inputs.noisy_density(32, 32, seed=2, mean=0.7, amp=0.05)
    with Lattice(rho0, G1=-400.0, G2=0.0, trace_every=1) as lat:
        lat.step(300)
        with pytest.raises(LBError) as ei:
            lat.trace()
        assert ei.value.status == capi.LB_ERR_NONFINITE


# ----------------------------------------------------------------- invariants on the GPU
def test_uniform_state_stays_exactly_uniform_gpu():
    for prec in ("fp32", "fp64", "fp16_delta"):
        rho0 = np.full((40, 64), 0.7)
        rho, ux, uy, tr, en = _run_gpu(rho0, 50, prec=prec, G1=-5.0, G2=0.6, trace_every=10)
        assert np.max(np.abs(rho - 0.7)) <= (1e-14 if prec == "fp64" else 1e-7)
        assert np.max(np.abs(ux)) <= 1e-15 and np.max(np.abs(uy)) <= 1e-15


def test_uniform_energy_closed_form_gpu():
    """Sec. 5: uniform psi gives E_s + E_m = E_bulk = A1/2 N psi^2, E_m = G2/2 N psi^2 596/15120."""
    psi = 1.0 - math.exp(-0.7)
    N = 40 * 64
    for prec, tol in (("fp64", 1e-13), ("fp32", 1e-6)):
        with Lattice(np.full((40, 64), 0.7), prec=prec, G1=-5.0, G2=0.6) as lat:
            es, em, eb, mass = lat.energy()
        assert abs(eb - (-4.4) / 2 * N * psi * psi) <= tol * abs(eb)
        assert abs(es + em - eb) <= tol * abs(eb)
        assert abs(em - 0.6 / 2 * N * psi * psi * 596 / 15120) <= tol * abs(em) + 1e-12
        assert abs(mass - 0.7 * N) <= tol * mass


def test_total_momentum_stays_zero_gpu():
    """sum_x F = 0 for the antisymmetric stencil, so sum rho u stays at its initial 0."""
    rho0 = inputs.noisy_density(96, 64, seed=21, mean=0.7, amp=0.05)
    for prec, tol in (("fp64", 1e-11), ("fp32", 1e-5)):
        rho, ux, uy, _, _ = _run_gpu(rho0, 300, prec=prec, G1=-5.0, G2=0.6, trace_every=0)
        assert rho.max() - rho.min() > 0.1
        assert abs((rho * ux).sum()) <= tol and abs((rho * uy).sum()) <= tol


def test_translation_is_exact_gpu():
    """Every site runs the same arithmetic whatever tile it falls in: a periodic shift of
    the input shifts the fields bit for bit (FP32 fused kernel, odd shape)."""
    rho0 = inputs.noisy_density(301, 77, seed=22, mean=0.7, amp=0.01, mode="rel")
    a = _run_gpu(rho0, 40, G1=-5.0, G2=0.6, trace_every=0, rho_ref=0.7)
    b = _run_gpu(np.roll(rho0, (5, -33), (0, 1)), 40, G1=-5.0, G2=0.6, trace_every=0, rho_ref=0.7)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(np.roll(u, (5, -33), (0, 1)), v)


def test_allocation_failure_returns_oom_and_cleans_up():
    rho0 = inputs.noisy_density(64, 64, seed=1)
    for after in (0, 3, 7):
        capi.lb_debug_fail_alloc(after)
        try:
            with pytest.raises(LBError) as ei:
                Lattice(rho0)
            assert ei.value.status == capi.LB_ERR_OOM
        finally:
            capi.lb_debug_fail_alloc(-1)
    # the library keeps working afterwards
    rho, _, _, _, _ = _run_gpu(rho0, 5, G1=-5.0, G2=0.0, trace_every=0)
    assert np.isfinite(rho).all()


def test_init_input_may_be_reused_at_once():
    """lb_init has read rho_init completely when it returns (one copy into the state,
    then a synchronisation; the initialisation itself runs on the stream): overwriting a
    device or pinned host rho_init right after lb_init leaves the state unchanged."""
    torch = pytest.importorskip("torch")
    rho0 = inputs.noisy_density(300, 200, seed=23, mean=0.7, amp=0.01, mode="rel")
    ref = _run_gpu(rho0, 20, G1=-5.0, G2=0.6, trace_every=0)
    for where in ("cuda", "pinned"):
        t = torch.from_numpy(rho0.copy())
        t = t.cuda() if where == "cuda" else t.pin_memory()
        with Lattice(t, G1=-5.0, G2=0.6, trace_every=0) as lat:
            t.fill_(5.0)                       # at once, before any step
            lat.step(20)
            got = lat.fields()
        for u, v in zip(got, ref[:3]):
            assert np.array_equal(u, v), where


@pytest.mark.parametrize("nx,ny,launch", [(130, 2000, (64, 4, 0)), (61, 997, (64, 5, 0)),
                                          (4000, 9, (256, 4, 0))])
def test_reduction_grid_sum_shapes(nx, ny, launch):
    """The reduction step's grid sum (one CTA per row of step CTAs, then the row totals)
    on grids of many short CTA rows (500 and 200 rows of 3 and 1 CTAs) and of few long ones
    (3 rows of 16 CTAs): trace and mass against the oracle, and the same trace bit for bit
    from a second run."""
    rho0 = inputs.noisy_density(nx, ny, seed=31, mean=0.7, amp=0.01, mode="rel")
    ref = oracle.run(rho0, 30, G1=-5.0, G2=0.6, trace_every=10)
    rho, ux, uy, tr, _ = _run_gpu(rho0, 30, launch=launch, G1=-5.0, G2=0.6, trace_every=10)
    assert len(tr) == 3 and np.array_equal(tr[:, 0], ref[3][:, 0])
    assert np.max(np.abs(tr[:, 1] - ref[3][:, 1]) / ref[3][:, 1]) <= 1e-6
    assert _trace_err(tr, ref[3]) <= 1e-4
    assert _norm_err(rho, ref[0]) <= 1e-5
    tr2 = _run_gpu(rho0, 30, launch=launch, G1=-5.0, G2=0.6, trace_every=10)[3]
    assert np.array_equal(tr, tr2)
