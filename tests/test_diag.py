"""Host-side observables (droplet count, perimeter, structure factor, radius)
on fields whose answers are known by construction."""
import math

import numpy as np

from paper_1008_2865_gb300 import diag


def _disk(L, cx, cy, r):
    y, x = np.mgrid[0:L, 0:L]
    dx = (x - cx + L / 2) % L - L / 2          # periodic distance
    dy = (y - cy + L / 2) % L - L / 2
    return dx * dx + dy * dy <= r * r


def test_droplets_periodic_merging():
    L = 64
    liq = _disk(L, 10, 10, 5) | _disk(L, 0, 40, 6) | _disk(L, 40, 63, 4)   # two wrap an edge
    rho = np.where(liq, 1.9, 0.15)
    n, lab = diag.droplets(rho)
    assert n == 3
    assert len(np.unique(lab[liq])) == 3 and np.all(lab[~liq] == 0)
    # a band across the whole lattice is one droplet; diagonal contact does not connect
    band = np.zeros((L, L), bool)
    band[20:25, :] = True
    assert diag.droplets(np.where(band, 1.9, 0.15))[0] == 1
    chk = np.zeros((8, 8), bool)
    chk[2, 2] = chk[3, 3] = True
    assert diag.droplets(np.where(chk, 1.9, 0.15))[0] == 2
    assert diag.droplets(np.full((8, 8), 0.15))[0] == 0


def test_perimeter_and_surface_to_volume():
    L = 50
    sq = np.zeros((L, L), bool)
    sq[10:22, 30:37] = True                      # 12 x 7 block
    rho = np.where(sq, 1.9, 0.15)
    assert diag.perimeter(rho) == 2 * (12 + 7)
    band = np.zeros((L, L), bool)
    band[:, 5:15] = True
    assert diag.perimeter(np.where(band, 1.9, 0.15)) == 2 * L
    assert diag.surface_to_volume(rho) == 2 * (12 + 7) / L ** 2


def test_structure_factor_peak_and_radius():
    L = 128
    x = np.arange(L)[None, :].repeat(L, 0)
    for m in (3, 10):
        rho = 0.7 + 0.01 * np.cos(2 * math.pi * m * x / L)
        n, Sk = diag.structure_factor(rho)
        assert int(np.argmax(Sk)) == m
        assert math.isclose(diag.radius(rho), L / (2 * m), rel_tol=1e-9)
        assert math.isclose(diag.radius(rho, literal=True), L / m, rel_tol=1e-9)


def test_thermal_energy_and_summary():
    rho = np.full((10, 10), 0.6)
    assert math.isclose(diag.thermal_energy(rho), 0.6 / 3 * 100)
    s = diag.summary(rho + 0.001 * np.cos(np.arange(10))[None, :], energies=(-2.0, -0.1, -2.2, 60.0))
    assert s["droplets"] == 0 and math.isclose(s["Em_over_Es"], 0.05)
    assert math.isclose(s["E_surface_share"], 0.1 / 2.2)
