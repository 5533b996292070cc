"""FP64 CPU oracle for the two-belt Shan–Chen D2Q9 lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY. Chibbaro et al., arXiv:1008.2865: Eq. 1 (LBE),
Eqs. 2-4 (moments, equilibrium), Eq. forza and Eq. FORCE with Table 1 (the
two-belt force), Sec. 5 (pseudo-energies). The arithmetic lives in
``lbsc_oracle.c`` (plain per-site loops, FP64, no contraction); this module
compiles it with gcc and wraps it with ctypes. Only the tests, the package
smoke check and the benchmark's CPU-baseline leg may import this package; the
CUDA library shares no code with it.

Pins (checked in ``tests/test_oracle_pins.py``): Table 1 weights and their
normalisations, the plane-wave Fourier symbol of the force against the
Taylor coefficients of Eq. ftot and the 8th-order isotropy claim, uniform
state invariance, mass and momentum conservation, D4 symmetry and
translation, the uniform-state energy closed form, the single-belt reduction
to Eq. forza, the critical coupling G_cr = -4, the linearised growth rate of
a Fourier mode, mechanical equilibrium across a flat interface, and a
40-digit brute-force step on a 5x5 lattice. Nothing here is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbsc_oracle.c")
_LIB = os.path.join(_HERE, "liblbsc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into an in-tree shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbsc_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
            "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm",
        ]
        if _needs_quadmath():
            cmd.append("-lquadmath")
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _needs_quadmath() -> bool:
    """True where long double is narrower than binary128 (x86): expq comes from libquadmath."""
    import platform
    return platform.machine() in ("x86_64", "AMD64", "i686")


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("omega", ctypes.c_double), ("G1", ctypes.c_double),
        ("G2", ctypes.c_double), ("rho0", ctypes.c_double),
    ]


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(_Params)
    lib.orc_threads.restype = ctypes.c_int
    lib.orc_link_table.argtypes = [ip, ip, dp, dp]
    lib.orc_psi.argtypes = [ctypes.c_long, dp, ctypes.c_double, dp]
    lib.orc_force.argtypes = [pp, dp, dp, dp]
    lib.orc_energy.argtypes = [pp, dp, dp]
    lib.orc_init.argtypes = [pp, dp, dp]
    lib.orc_moments.argtypes = [pp, dp, dp, dp, dp]
    lib.orc_step.argtypes = [pp, dp, dp]
    lib.orc_run.argtypes = [pp, dp, ctypes.c_long, ctypes.c_int, dp, dp, dp,
                            dp, ctypes.c_int, ip]
    lib.orc_run.restype = ctypes.c_int
    lib.orc_objective.argtypes = [pp, dp, ctypes.c_long, dp, dp]
    lib.orc_objective.restype = ctypes.c_double
    lib.orc_gradient.argtypes = [pp, dp, ctypes.c_long, dp, dp, dp, dp]
    lib.orc_gradient.restype = ctypes.c_int
    lib.orc_adjoint_step.argtypes = [pp, dp, dp, dp, dp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class use_library:
    """Context manager that points this module at another build of the oracle
    source (the mutation tests compile deliberately broken copies)."""

    def __init__(self, path):
        self.lib = _bind(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        _lib = self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def compile_source(src_text: str, out_path: str) -> str:
    """Compile oracle C source text (same flags as build()) into out_path."""
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "lbsc_oracle.c")
        with open(c, "w") as fh:
            fh.write(src_text)
        import shutil
        shutil.copy(os.path.join(_HERE, "lbsc_oracle.h"), td)
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-fPIC", "-shared", c, "-o", out_path, "-lm"]
        if _needs_quadmath():
            cmd.append("-lquadmath")
        subprocess.run(cmd, check=True)
    return out_path


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(nx, ny, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0):
    return _Params(int(nx), int(ny), float(omega), float(G1), float(G2), float(rho0))


def threads() -> int:
    """OpenMP threads the oracle runs on."""
    return int(_load().orc_threads())


def link_table():
    """(cx, cy, w, p) for the rest link, the 8 belt-1 links and the 16 belt-2 links."""
    lib = _load()
    cx = np.zeros(25, np.int32)
    cy = np.zeros(25, np.int32)
    w = np.zeros(25)
    p = np.zeros(25)
    lib.orc_link_table(cx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       cy.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w), _dp(p))
    return cx, cy, w, p


def psi(rho, rho0=1.0):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    _load().orc_psi(rho.size, _dp(rho), float(rho0), _dp(out))
    return out


def force(psi_field, G1, G2):
    """Two-belt force (Fx, Fy) of a periodic psi field shaped [ny, nx]."""
    ps = np.ascontiguousarray(psi_field, dtype=np.float64)
    ny, nx = ps.shape
    fx = np.empty_like(ps)
    fy = np.empty_like(ps)
    P = _params(nx, ny, G1=G1, G2=G2)
    _load().orc_force(ctypes.byref(P), _dp(ps), _dp(fx), _dp(fy))
    return fx, fy


def energy(psi_field, G1, G2):
    """(E_s, E_m, E_bulk) of a periodic psi field shaped [ny, nx]."""
    ps = np.ascontiguousarray(psi_field, dtype=np.float64)
    ny, nx = ps.shape
    out = np.empty(3)
    P = _params(nx, ny, G1=G1, G2=G2)
    _load().orc_energy(ctypes.byref(P), _dp(ps), _dp(out))
    return tuple(float(v) for v in out)


def init(rho, **kw):
    """f_i = w_i rho, shaped [9, ny, nx]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    f = np.empty((9, ny, nx))
    P = _params(nx, ny, **kw)
    _load().orc_init(ctypes.byref(P), _dp(rho), _dp(f))
    return f


def moments(f):
    """(rho, ux, uy) of populations shaped [9, ny, nx]."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    rho = np.empty((ny, nx))
    ux = np.empty((ny, nx))
    uy = np.empty((ny, nx))
    P = _params(nx, ny)
    _load().orc_moments(ctypes.byref(P), _dp(f), _dp(rho), _dp(ux), _dp(uy))
    return rho, ux, uy


def step(f, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0):
    """One step of Eq. 1 on populations shaped [9, ny, nx]; returns the new f."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    P = _params(nx, ny, omega, G1, G2, rho0)
    _load().orc_step(ctypes.byref(P), _dp(f), _dp(out))
    return out


def run(rho_init, steps, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0, trace_every=0,
        trace_cap=None):
    """Run `steps` steps from f = w rho_init.

    Returns (rho, ux, uy, trace) with trace an array of rows
    (t, mass, E_s, E_m, E_bulk) for t < steps, t % trace_every == 0.
    """
    rho_init = np.ascontiguousarray(rho_init, dtype=np.float64)
    ny, nx = rho_init.shape
    rho = np.empty((ny, nx))
    ux = np.empty((ny, nx))
    uy = np.empty((ny, nx))
    if trace_every and trace_every > 0:
        cap = trace_cap if trace_cap is not None else (steps + trace_every - 1) // trace_every
        cap = max(int(cap), 1)
    else:
        cap = 1
    trace = np.zeros((cap, 5))
    count = ctypes.c_int(0)
    P = _params(nx, ny, omega, G1, G2, rho0)
    rc = _load().orc_run(ctypes.byref(P), _dp(rho_init), int(steps), int(trace_every or 0),
                         _dp(rho), _dp(ux), _dp(uy), _dp(trace), cap, ctypes.byref(count))
    if rc != 0:
        raise ValueError("oracle rejected the parameters or ran out of memory")
    return rho, ux, uy, trace[: count.value].copy()


def objective(rho_init, rho_target, steps, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0):
    """(J, E) with J = E_s(T) + E_m(T) + sum (rho(T) - rho_target)^2."""
    rho_init = np.ascontiguousarray(rho_init, dtype=np.float64)
    tgt = np.ascontiguousarray(rho_target, dtype=np.float64)
    ny, nx = rho_init.shape
    E = ctypes.c_double(0.0)
    P = _params(nx, ny, omega, G1, G2, rho0)
    J = _load().orc_objective(ctypes.byref(P), _dp(rho_init), int(steps), _dp(tgt),
                              ctypes.byref(E))
    return float(J), float(E.value)


def gradient(rho_init, rho_target, steps, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0):
    """(J, dJ/drho_init [ny, nx], (dJ/dG1, dJ/dG2)) by the reverse sweep."""
    rho_init = np.ascontiguousarray(rho_init, dtype=np.float64)
    tgt = np.ascontiguousarray(rho_target, dtype=np.float64)
    ny, nx = rho_init.shape
    g = np.empty((ny, nx))
    gG = np.empty(2)
    J = ctypes.c_double(0.0)
    P = _params(nx, ny, omega, G1, G2, rho0)
    if _load().orc_gradient(ctypes.byref(P), _dp(rho_init), int(steps), _dp(tgt),
                            ctypes.byref(J), _dp(g), _dp(gG)) != 0:
        raise ValueError("oracle rejected the parameters or ran out of memory")
    return float(J.value), g, (float(gG[0]), float(gG[1]))


def adjoint_step(f, lam_next, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0):
    """(lam, (gG1, gG2)): the transpose of one step's Jacobian at f applied to lam_next."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    ln = np.ascontiguousarray(lam_next, dtype=np.float64)
    _, ny, nx = f.shape
    lam = np.empty_like(f)
    gG = np.empty(2)
    P = _params(nx, ny, omega, G1, G2, rho0)
    _load().orc_adjoint_step(ctypes.byref(P), _dp(f), _dp(ln), _dp(lam), _dp(gG))
    return lam, (float(gG[0]), float(gG[1]))
