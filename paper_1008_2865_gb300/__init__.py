"""GB300-native two-belt Shan–Chen lattice Boltzmann (Chibbaro et al., arXiv:1008.2865).

The compute path is liblbsc.so (CUDA, sm_103a) behind the C ABI of
include/lb.h; :mod:`paper_1008_2865_gb300.capi` binds it with ctypes under the
same names, and :class:`Lattice` wraps one state. PyTorch, when used, only
supplies device memory and the CUDA stream.
"""
from __future__ import annotations

import numpy as np

from . import capi, inputs  # noqa: F401
from .capi import (lb_batch_count, lb_batch_destroy, lb_batch_energy, lb_batch_fields,  # noqa: F401
                   lb_batch_get_launch, lb_batch_init, lb_batch_set_launch, lb_batch_step,
                   lb_batch_time, lb_batch_trace)
from .capi import (lb_adjoint, lb_load_state, lb_objective, lb_save_state,  # noqa: F401
                   lb_state_bytes)
from .capi import (LBError, lb_destroy, lb_energy, lb_fields, lb_get_launch,  # noqa: F401
                   lb_init, lb_set_launch, lb_set_wait_limit, lb_status_str, lb_step, lb_time,
                   lb_trace, make_params)


def couplings_from_A(A1: float, A2: float, lam: float = 1.5):
    """(G1, G2) from the Sec. 4 parameters A1 = G1 + G2 and A2 = G1 + lam G2 (lam = 3/2)."""
    G2 = (A2 - A1) / (lam - 1.0)
    return A1 - G2, G2


class Lattice:
    """One periodic lattice on the GPU.

    >>> lat = Lattice(rho_init, G1=-5.0, G2=0.6)        # rho_init: [ny, nx] float64
    >>> lat.step(100); E_s, E_m, E_bulk, mass = lat.energy()
    """

    def __init__(self, rho_init, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0, prec="fp32",
                 trace_every=10, rho_ref=0.0, device=0, stream=0):
        ny, nx = rho_init.shape
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(nx, ny, omega, G1, G2, rho0, prec, trace_every, rho_ref, device)
        self.handle = lb_init(self.params, rho_init, stream)

    def step(self, n: int = 1) -> None:
        lb_step(self.handle, n)

    @property
    def t(self) -> int:
        return lb_time(self.handle)

    def energy(self):
        return lb_energy(self.handle)

    def fields(self, rho=None, ux=None, uy=None):
        """Fill the given [ny, nx] float64 arrays/tensors; with none given, return NumPy arrays."""
        if rho is None and ux is None and uy is None:
            rho = np.empty((self.ny, self.nx))
            ux = np.empty((self.ny, self.nx))
            uy = np.empty((self.ny, self.nx))
            lb_fields(self.handle, rho, ux, uy)
            return rho, ux, uy
        lb_fields(self.handle, rho, ux, uy)
        return rho, ux, uy

    def save(self, dst=None):
        """The state in its saved form (NumPy uint8 buffer unless dst is given)."""
        return lb_save_state(self.handle, dst)

    def load(self, src) -> None:
        """Resume from a saved form (same size, precision and reference density)."""
        lb_load_state(self.handle, src)

    def adjoint(self, steps: int, rho_target, checkpoint_every: int = 0, grad_rho=None):
        """(J, dJ/drho_init, (dJ/dG1, dJ/dG2)) of J = E_s(T) + E_m(T) + sum (rho(T) - rho*)^2
        over `steps` steps from this (fresh, FP32) state; leaves the state at t = steps."""
        return lb_adjoint(self.handle, steps, rho_target, checkpoint_every, grad_rho)

    def objective(self, rho_target) -> float:
        """J = E_s + E_m + sum (rho - rho*)^2 of the current state (the adjoint's objective)."""
        return lb_objective(self.handle, rho_target)

    @property
    def launch(self):
        """(block_x, rows_per_cta, pipeline) of the fused step kernel."""
        return lb_get_launch(self.handle)

    def set_launch(self, block_x: int, rows_per_cta: int, pipeline: int = None) -> None:
        if pipeline is None:
            pipeline = self.launch[2]
        lb_set_launch(self.handle, block_x, rows_per_cta, pipeline)

    def trace(self, cap: int = 65536):
        return lb_trace(self.handle, cap)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent lattices advanced together (one launch per step for all).

    >>> b = Batch([rho_a, rho_b], G2=[0.3, 0.6])      # per-replica values or scalars
    >>> b.step(100); rho, ux, uy = b.fields(1)
    """

    def __init__(self, rho_list, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0, prec="fp32",
                 trace_every=10, rho_ref=0.0, device=0, stream=0):
        n = len(rho_list)

        def per(v):
            return list(v) if isinstance(v, (list, tuple, np.ndarray)) else [v] * n

        om, g1, g2, r0, rr = per(omega), per(G1), per(G2), per(rho0), per(rho_ref)
        self.shapes = [tuple(r.shape) for r in rho_list]
        params = [make_params(r.shape[1], r.shape[0], om[i], g1[i], g2[i], r0[i], prec,
                              trace_every, rr[i], device) for i, r in enumerate(rho_list)]
        self.handle = lb_batch_init(params, rho_list, stream)

    def __len__(self):
        return lb_batch_count(self.handle)

    @property
    def t(self) -> int:
        return lb_batch_time(self.handle)

    def step(self, n: int = 1) -> None:
        lb_batch_step(self.handle, n)

    def energy(self, i: int):
        return lb_batch_energy(self.handle, i)

    def fields(self, i: int, rho=None, ux=None, uy=None):
        if rho is None and ux is None and uy is None:
            ny, nx = self.shapes[i]
            rho, ux, uy = np.empty((ny, nx)), np.empty((ny, nx)), np.empty((ny, nx))
        lb_batch_fields(self.handle, i, rho, ux, uy)
        return rho, ux, uy

    def trace(self, i: int, cap: int = 65536):
        return lb_batch_trace(self.handle, i, cap)

    @property
    def launch(self):
        return lb_batch_get_launch(self.handle)

    def set_launch(self, block_x: int, rows_per_cta: int, use_graph: int = 1) -> None:
        lb_batch_set_launch(self.handle, block_x, rows_per_cta, use_graph)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
