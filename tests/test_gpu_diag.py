"""The paper's observables from GPU runs against the same observables computed from
the oracle's fields (Sec. 4 radius and droplets, Sec. 5 energy series and E_surf,
Eq. gamma on a flat interface). The FP64 path follows the oracle bit for bit, so
its observables must be identical; the FP32 path within the stated tolerances."""
import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import Lattice, diag, inputs

pytestmark = pytest.mark.gpu

G1, G2 = -5.0, 0.5


def _series_gpu(prec, rho0, marks, trace_every=10):
    snaps = {}
    with Lattice(rho0, G1=G1, G2=G2, prec=prec, trace_every=trace_every) as lat:
        done = 0
        for m in marks:
            lat.step(m - done)
            done = m
            snaps[m] = lat.fields()[0]
        tr = lat.trace()
    return snaps, tr


def _observables(rho):
    return {"R": diag.radius(rho), "droplets": diag.droplets(rho)[0],
            "S/V": diag.surface_to_volume(rho), "E_surf": diag.surface_energy(rho, G1, G2)}


def test_time_series_match_the_oracle():
    n, marks = 64, (200, 400, 600)
    rho0 = inputs.noisy_density(n, n, 31, mean=0.7, amp=0.01, mode="rel")
    ref = {m: oracle.run(rho0, m, G1=G1, G2=G2)[0] for m in marks}
    ref_trace = oracle.run(rho0, marks[-1], G1=G1, G2=G2, trace_every=10)[3]
    s_ref = diag.energy_series(ref_trace, n * n)
    for prec in ("fp64", "fp32"):
        snaps, tr = _series_gpu(prec, rho0, marks)
        s = diag.energy_series(tr, n * n)
        assert np.array_equal(s["t"], s_ref["t"])
        # the GPU's FP64 energy sums add the same site terms as the oracle in another
        # order (rounding 1e-16 of E); the surface share is a small difference of two
        # such sums, so it is compared absolutely, the ratios relatively
        for key in ("E_over_Eth", "Em_over_Es"):
            tol = 1e-12 if prec == "fp64" else 1e-4
            assert np.max(np.abs(s[key] - s_ref[key]) / np.abs(s_ref[key])) <= tol, (prec, key)
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert np.max(np.abs(s["surface_share"] - s_ref["surface_share"])) <= tol, prec
        for m in marks:
            got, want = _observables(snaps[m]), _observables(ref[m])
            if prec == "fp64":
                assert got == want
            else:
                assert got["droplets"] == want["droplets"]
                assert abs(got["R"] - want["R"]) <= 1e-3 * want["R"]
                assert abs(got["S/V"] - want["S/V"]) <= 1e-2 * want["S/V"]
                assert abs(got["E_surf"] - want["E_surf"]) <= 1e-3 * abs(want["E_surf"])


def test_flat_interface_surface_tension_matches_the_oracle():
    """Eq. gamma on the y-averaged psi profile of a relaxed slab (64 x 5, 20000 steps):
    FP32 GPU against the oracle's FP64 fields to 1e-3."""
    nx, ny = 64, 5
    x = np.arange(nx) + 0.5
    prof = 0.155 + (1.93 - 0.155) * 0.5 * (np.tanh((x - 16) / 3) - np.tanh((x - 48) / 3))
    rho0 = np.ascontiguousarray(prof[None, :].repeat(ny, 0))
    ref = oracle.run(rho0, 20000, G1=-5.0, G2=0.0)[0]
    with Lattice(rho0, G1=-5.0, G2=0.0, trace_every=0) as lat:
        lat.step(20000)
        rho = lat.fields()[0]
    g_ref = diag.surface_tension(diag.psi_of(ref.mean(axis=0)), -5.0, 0.0)
    g = diag.surface_tension(diag.psi_of(rho.mean(axis=0)), -5.0, 0.0)
    assert g_ref > 0
    assert abs(g - g_ref) <= 1e-3 * g_ref
