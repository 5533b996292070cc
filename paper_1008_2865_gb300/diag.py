"""Observables of a density field, as the paper measures them (host-side post-processing).

- droplets(rho): connected liquid regions of a periodic lattice — liquid means
  rho > rho_th with rho_th = rho0 ln 2, the critical density (Sec. 2); sites
  are joined by their four nearest neighbours, across the periodic edges too.
- perimeter(rho): liquid-gas interface length in lattice units, the number of
  nearest-neighbour bonds joining a liquid and a gas site; surface/volume is
  perimeter / N ("perimeter in 2D" against the volume L^2, Sec. 5).
- structure_factor(rho): S(k) = |sum_x (rho - mean) e^{i k.x}|^2 / N on the
  discrete wave vectors, averaged over circular shells n - 1/2 <= |k| L / 2 pi
  < n + 1/2 (Sec. 4, Eq. rad).
- radius(rho): the typical domain size from the first moment of S(k): with
  n_bar = sum_n n S(n) / sum_n S(n), R = L / (2 n_bar) (Sec. 4: "k = 1 means
  R = L/2"); radius(..., literal=True) gives 2 pi / k_bar instead.
- thermal_energy(rho): E_th = rho_mean cs^2 L^2 (Sec. 5, Fig. 5).
- summary(rho, energies): the above plus E/E_th, E_m/E_s and the surface share
  (E - E_bulk) / |E_bulk| of the pseudo-energy (Sec. 5, Figs. 5 and 7).
- energy_series(trace, n_sites): the time series of Figs. 5 and 7 from the
  library's trace rows (t, mass, E_s, E_m, E_bulk): E/E_th, E_m/E_s and the
  surface share, with E_th = rho_mean cs^2 N and rho_mean = mass / N.
- growth_exponent(t, R, t0): the exponent alpha of R(t) ~ (t - t0)^alpha
  (Sec. 4: 1/3 for diffusive growth, 1/6 and 1/5 for the slowed cases) by a
  least-squares fit of log R against log(t - t0).
- surface_energy(rho, G1, G2): E_surf of Sec. 5 (Eq. Esurf) in weak-gradient
  form, c sum_x |grad psi|^2 with central differences on the periodic lattice;
  c = -A1/12 (the second-order expansion of the Sec. 5 sums under the
  normalisations of Eqs. weights_1 and weights_2, A1 = G1 + G2) by default,
  or c = A2/2 as printed (A2 = G1 + 3/2 G2) with coefficient="printed".
- surface_tension(psi_profile, G1, G2): gamma of Eq. gamma per interface,
  -(G1 + 12/7 G2)/2 cs^4 integral |d psi/dy|^2 dy, on a periodic profile across
  a flat slab (two interfaces; the integral is halved), central differences,
  unit lattice spacing.

Densities are NumPy arrays [ny, nx] (row-major [y][x]); nothing here is on the
GPU path. The FFT is NumPy's.
"""
from __future__ import annotations

import math

import numpy as np

CS2 = 1.0 / 3.0


def liquid_threshold(rho0: float = 1.0) -> float:
    """The critical density rho0 ln 2 (Sec. 2), used to tell liquid from gas."""
    return rho0 * math.log(2.0)


def _find(parent, a):
    while parent[a] != a:
        parent[a] = parent[parent[a]]
        a = parent[a]
    return a


def droplets(rho, threshold=None, liquid_above=True):
    """(count, labels): 4-connected liquid regions of a periodic lattice.

    labels is an int array [ny, nx] with 0 for gas and 1..count for liquid regions.
    """
    from scipy import ndimage

    th = liquid_threshold() if threshold is None else threshold
    liquid = rho > th if liquid_above else rho < th
    lab, n = ndimage.label(liquid, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    if n == 0:
        return 0, lab
    parent = list(range(n + 1))

    def union(a, b):
        ra, rb = _find(parent, a), _find(parent, b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)

    # periodic edges: left-right and top-bottom neighbours that are both liquid
    for a, b in zip(lab[:, 0], lab[:, -1]):
        if a and b:
            union(int(a), int(b))
    for a, b in zip(lab[0, :], lab[-1, :]):
        if a and b:
            union(int(a), int(b))
    roots = sorted({_find(parent, k) for k in range(1, n + 1)})
    remap = np.zeros(n + 1, dtype=np.int64)
    index = {r: i + 1 for i, r in enumerate(roots)}
    for k in range(1, n + 1):
        remap[k] = index[_find(parent, k)]
    return len(roots), remap[lab]


def perimeter(rho, threshold=None):
    """Number of nearest-neighbour liquid-gas bonds on the periodic lattice."""
    th = liquid_threshold() if threshold is None else threshold
    liq = rho > th
    return int(np.count_nonzero(liq != np.roll(liq, 1, axis=0)) +
               np.count_nonzero(liq != np.roll(liq, 1, axis=1)))


def surface_to_volume(rho, threshold=None):
    """perimeter / N."""
    return perimeter(rho, threshold) / rho.size


def structure_factor(rho):
    """(n, S(n)): the circularly averaged structure factor on shells n = 0, 1, ...

    Requires a square lattice (the shells are defined with one L)."""
    ny, nx = rho.shape
    if nx != ny:
        raise ValueError("circular shells need a square lattice")
    L = nx
    d = rho - rho.mean()
    S = np.abs(np.fft.fft2(d)) ** 2 / rho.size
    m = np.fft.fftfreq(L, d=1.0 / L)            # integer wave numbers -L/2 .. L/2 - 1
    kk = np.sqrt(m[None, :] ** 2 + m[:, None] ** 2)
    shell = np.floor(kk + 0.5).astype(np.int64)  # n - 1/2 <= |k| L / 2pi < n + 1/2
    nmax = L // 2
    sel = shell <= nmax
    sums = np.bincount(shell[sel], weights=S[sel], minlength=nmax + 1)
    counts = np.bincount(shell[sel], minlength=nmax + 1)
    n = np.arange(nmax + 1)
    Sk = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
    return n, Sk


def radius(rho, literal=False):
    """Typical domain size from the first moment of the circularly averaged S(k)."""
    n, Sk = structure_factor(rho)
    n, Sk = n[1:], Sk[1:]                        # the k = 0 shell carries no structure
    tot = Sk.sum()
    if tot <= 0:
        return float("inf")
    nbar = (n * Sk).sum() / tot
    L = rho.shape[0]
    if literal:
        return 2.0 * math.pi / (2.0 * math.pi * nbar / L)
    return L / (2.0 * nbar)


def thermal_energy(rho):
    """E_th = rho_mean cs^2 L^2 (Sec. 5)."""
    return float(rho.mean()) * CS2 * rho.size


def summary(rho, energies=None):
    """A dict of the observables of one density field (energies = (E_s, E_m, E_bulk, mass))."""
    count, _ = droplets(rho)
    out = {"droplets": count, "surface_to_volume": surface_to_volume(rho),
           "radius": radius(rho), "rho_min": float(rho.min()), "rho_max": float(rho.max())}
    if energies is not None:
        es, em, eb, _ = energies
        E = es + em
        out.update({"E_over_Eth": E / thermal_energy(rho), "Em_over_Es": em / es,
                    "E_surface_share": (E - eb) / abs(eb) if eb != 0 else 0.0})
    return out


def psi_of(rho, rho0: float = 1.0):
    """psi = sqrt(rho0) (1 - exp(-rho / rho0)) (Sec. 2)."""
    return math.sqrt(rho0) * -np.expm1(-np.asarray(rho, dtype=np.float64) / rho0)


def energy_series(trace, n_sites: int):
    """Figs. 5 and 7 from trace rows (t, mass, E_s, E_m, E_bulk): a dict of arrays
    t, E_over_Eth, Em_over_Es, surface_share ((E - E_bulk) / |E_bulk|)."""
    tr = np.asarray(trace, dtype=np.float64).reshape(-1, 5)
    t, mass, es, em, eb = (tr[:, k] for k in range(5))
    e = es + em
    eth = (mass / n_sites) * CS2 * n_sites
    with np.errstate(divide="ignore", invalid="ignore"):
        return {"t": t, "E_over_Eth": e / eth, "Em_over_Es": em / es,
                "surface_share": (e - eb) / np.abs(eb)}


def growth_exponent(t, R, t0: float = 0.0):
    """alpha of R(t) ~ (t - t0)^alpha: least-squares slope of log R on log(t - t0)."""
    t = np.asarray(t, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    sel = (t > t0) & np.isfinite(R) & (R > 0)
    if np.count_nonzero(sel) < 2:
        return float("nan")
    x = np.log(t[sel] - t0)
    y = np.log(R[sel])
    return float(np.polyfit(x, y, 1)[0])


def _grad_sq(psi):
    """|grad psi|^2 by central differences on the periodic lattice."""
    gx = 0.5 * (np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1))
    gy = 0.5 * (np.roll(psi, -1, axis=0) - np.roll(psi, 1, axis=0))
    return gx * gx + gy * gy


def surface_energy(rho, G1: float, G2: float, rho0: float = 1.0, coefficient: str = "expansion",
                   lam: float = 1.5):
    """E_surf = c sum_x |grad psi|^2 (Eq. Esurf), c = -A1/12 ("expansion") or A2/2
    ("printed", A2 = G1 + lam G2)."""
    psi = psi_of(rho, rho0)
    if coefficient == "expansion":
        c = -(G1 + G2) / 12.0
    elif coefficient == "printed":
        c = (G1 + lam * G2) / 2.0
    else:
        raise ValueError(f"unknown coefficient {coefficient!r}")
    return float(c * _grad_sq(psi).sum())


def surface_tension(psi_profile, G1: float, G2: float, interfaces: int = 2):
    """gamma of Eq. gamma for each of the `interfaces` interfaces of a periodic
    profile psi(y) across a flat slab: -(G1 + 12/7 G2)/2 cs^4 sum_y (d psi/dy)^2 / interfaces."""
    p = np.asarray(psi_profile, dtype=np.float64)
    d = 0.5 * (np.roll(p, -1) - np.roll(p, 1))
    return float(-(G1 + 12.0 / 7.0 * G2) / 2.0 * CS2 * CS2 * np.sum(d * d) / interfaces)
