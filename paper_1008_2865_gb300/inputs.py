"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle's tests.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
turns (seed, site index) into uniform random numbers and those into initial
density fields of the kind Sec. 4 of the paper describes (a noisy uniform
density on a periodic box).

Uniform variates come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the 64-bit input for site k is (seed << 32) XOR k, it is mixed by
one SplitMix64 output step, and the top 53 bits of the result, divided by
2**53, give U in [0, 1).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """One SplitMix64 output step applied elementwise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in [0, 1) for site indices offset .. offset+n-1 (FP64)."""
    k = np.arange(offset, offset + n, dtype=np.uint64)
    x = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) ^ k
    z = splitmix64(x)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def noisy_density(nx: int, ny: int, seed: int, mean: float = 0.7, amp: float = 0.01,
                  mode: str = "abs") -> np.ndarray:
    """Initial density [ny, nx] (row-major [y][x]), FP64.

    mode "abs": rho = mean + amp * (2U - 1)       (uniform noise of half-width amp)
    mode "rel": rho = mean * (1 + amp * (2U - 1)) (relative noise, "±1%" for amp=0.01)
    """
    u = uniform(seed, nx * ny).reshape(ny, nx)
    if mode == "abs":
        return mean + amp * (2.0 * u - 1.0)
    if mode == "rel":
        return mean * (1.0 + amp * (2.0 * u - 1.0))
    raise ValueError(f"unknown noise mode {mode!r}")


def noisy_density_rows(nx: int, y0: int, y1: int, seed: int, mean: float = 0.7,
                       amp: float = 0.01, mode: str = "abs") -> np.ndarray:
    """Rows y0..y1-1 of the field noisy_density(nx, ny, seed, ...) would give (any ny > y1)."""
    u = uniform(seed, nx * (y1 - y0), offset=nx * y0).reshape(y1 - y0, nx)
    if mode == "abs":
        return mean + amp * (2.0 * u - 1.0)
    if mode == "rel":
        return mean * (1.0 + amp * (2.0 * u - 1.0))
    raise ValueError(f"unknown noise mode {mode!r}")


def g2_sweep(count: int, seed: int = 100, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """count couplings G2 drawn uniformly in [lo, hi) (a batched parameter sweep)."""
    return lo + (hi - lo) * uniform(seed, count)
