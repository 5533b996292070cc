"""ctypes binding of liblbsc.so — the functions of include/lb.h under the same names.

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels. There is no fallback: if the shared library is
missing or cannot be loaded, every call raises.

Pointers may be NumPy arrays (host memory) or anything exposing
``data_ptr()`` (torch tensors on the state's device). Streams are passed as
the integer handle ``torch.cuda.Stream.cuda_stream`` (0 = legacy default).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_OOM, LB_ERR_NONFINITE, LB_ERR_STATE = 0, -1, -2, -3, -4, -5
LB_ERR_TIMEOUT = -6
LB_PSI_SC_EXP = 0
LB_FP32, LB_FP64, LB_FP16_DELTA = 0, 1, 2

_PRECISION = {"fp32": LB_FP32, "fp64": LB_FP64, "fp16_delta": LB_FP16_DELTA}


class lb_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("omega", ctypes.c_double), ("G1", ctypes.c_double), ("G2", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("psi_form", ctypes.c_int), ("prec", ctypes.c_int), ("trace_every", ctypes.c_int),
        ("rho_ref", ctypes.c_double), ("device", ctypes.c_int),
    ]


class LBError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lb_status_str(status)} ({status})")


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblbsc.so (building it first only when asked)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(
                        f"{path} is missing: build it with paper_1008_2865_gb300.build.build()")
                _build.build()
            lib = ctypes.CDLL(path)
            vp = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            lib.lb_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(lb_params), vp, vp]
            lib.lb_init.restype = ctypes.c_int
            lib.lb_step.argtypes = [vp, ctypes.c_long]
            lib.lb_step.restype = ctypes.c_int
            lib.lb_energy.argtypes = [vp, dp]
            lib.lb_energy.restype = ctypes.c_int
            lib.lb_fields.argtypes = [vp, vp, vp, vp]
            lib.lb_fields.restype = ctypes.c_int
            lib.lb_trace.argtypes = [vp, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.lb_trace.restype = ctypes.c_int
            lib.lb_time.argtypes = [vp]
            lib.lb_time.restype = ctypes.c_long
            ip = ctypes.POINTER(ctypes.c_int)
            lib.lb_get_launch.argtypes = [vp, ip, ip, ip]
            lib.lb_get_launch.restype = ctypes.c_int
            lib.lb_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.lb_set_launch.restype = ctypes.c_int
            lib.lb_set_wait_limit.argtypes = [vp, ctypes.c_longlong, ctypes.c_int]
            lib.lb_set_wait_limit.restype = ctypes.c_int
            lib.lb_batch_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int,
                                          ctypes.POINTER(lb_params), ctypes.POINTER(vp), vp]
            lib.lb_batch_init.restype = ctypes.c_int
            lib.lb_batch_step.argtypes = [vp, ctypes.c_long]
            lib.lb_batch_step.restype = ctypes.c_int
            lib.lb_batch_energy.argtypes = [vp, ctypes.c_int, dp]
            lib.lb_batch_energy.restype = ctypes.c_int
            lib.lb_batch_fields.argtypes = [vp, ctypes.c_int, vp, vp, vp]
            lib.lb_batch_fields.restype = ctypes.c_int
            lib.lb_batch_trace.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
            lib.lb_batch_trace.restype = ctypes.c_int
            lib.lb_batch_get_launch.argtypes = [vp, ip, ip, ip]
            lib.lb_batch_get_launch.restype = ctypes.c_int
            lib.lb_batch_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.lb_batch_set_launch.restype = ctypes.c_int
            lib.lb_batch_check_guards.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
            lib.lb_batch_check_guards.restype = ctypes.c_int
            lib.lb_batch_count.argtypes = [vp]
            lib.lb_batch_count.restype = ctypes.c_int
            lib.lb_batch_time.argtypes = [vp]
            lib.lb_batch_time.restype = ctypes.c_long
            lib.lb_batch_destroy.argtypes = [vp]
            lib.lb_batch_destroy.restype = None
            lib.lb_check_guards.argtypes = [vp, ip]
            lib.lb_check_guards.restype = ctypes.c_int
            lib.lb_debug_fail_alloc.argtypes = [ctypes.c_int]
            lib.lb_debug_fail_alloc.restype = None
            lib.lb_debug_damage_guard.argtypes = [vp, ctypes.c_int]
            lib.lb_debug_damage_guard.restype = ctypes.c_int
            lib.lb_state_bytes.argtypes = [vp]
            lib.lb_state_bytes.restype = ctypes.c_size_t
            lib.lb_save_state.argtypes = [vp, vp, ctypes.c_size_t]
            lib.lb_save_state.restype = ctypes.c_int
            lib.lb_load_state.argtypes = [vp, vp, ctypes.c_size_t]
            lib.lb_load_state.restype = ctypes.c_int
            lib.lb_adjoint.argtypes = [vp, ctypes.c_long, vp, ctypes.c_int, dp, vp, dp]
            lib.lb_adjoint.restype = ctypes.c_int
            lib.lb_objective.argtypes = [vp, vp, dp]
            lib.lb_objective.restype = ctypes.c_int
            lib.lb_energy_noalloc.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, ctypes.c_double, vp, vp]
            lib.lb_energy_noalloc.restype = ctypes.c_int
            lib.lb_destroy.argtypes = [vp]
            lib.lb_destroy.restype = None
            lib.lb_status_str.argtypes = [ctypes.c_int]
            lib.lb_status_str.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def _ptr(a):
    """Raw address of a NumPy array / torch tensor / int / None."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot pass {type(a)!r} as a pointer")


def _check(st: int, where: str):
    if st != LB_OK:
        raise LBError(st, where)


def make_params(nx, ny, omega=1.0, G1=-5.0, G2=0.0, rho0=1.0, prec="fp32", trace_every=10,
                rho_ref=0.0, device=0, psi_form=LB_PSI_SC_EXP) -> lb_params:
    return lb_params(int(nx), int(ny), float(omega), float(G1), float(G2), float(rho0),
                     int(psi_form), _PRECISION.get(prec, prec), int(trace_every),
                     float(rho_ref), int(device))


def lb_status_str(st: int) -> str:
    return load().lb_status_str(int(st)).decode()


def lb_init(params: lb_params, rho_init, stream: int = 0) -> int:
    """Returns the opaque state handle (an int). rho_init: [ny, nx] float64, host or device."""
    if isinstance(rho_init, np.ndarray):
        rho_init = np.ascontiguousarray(rho_init, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load().lb_init(ctypes.byref(h), ctypes.byref(params), _ptr(rho_init),
                          ctypes.c_void_p(stream or None)), "lb_init")
    return h.value


def lb_step(h: int, n: int) -> None:
    _check(load().lb_step(ctypes.c_void_p(h), int(n)), "lb_step")


def lb_energy(h: int):
    """(E_s, E_m, E_bulk, mass) of the current state."""
    out = (ctypes.c_double * 4)()
    st = load().lb_energy(ctypes.c_void_p(h), out)
    if st not in (LB_OK, LB_ERR_NONFINITE):
        raise LBError(st, "lb_energy")
    vals = tuple(out)
    if st == LB_ERR_NONFINITE:
        raise LBError(st, f"lb_energy {vals}")
    return vals


def lb_fields(h: int, rho=None, ux=None, uy=None) -> None:
    _check(load().lb_fields(ctypes.c_void_p(h), _ptr(rho), _ptr(ux), _ptr(uy)), "lb_fields")


def lb_trace(h: int, cap: int = 65536) -> np.ndarray:
    buf = np.zeros((max(cap, 1), 5))
    cnt = ctypes.c_int(0)
    _check(load().lb_trace(ctypes.c_void_p(h), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           int(cap), ctypes.byref(cnt)), "lb_trace")
    return buf[: cnt.value].copy()


def lb_get_launch(h: int):
    """(block_x, rows_per_cta, pipeline) of the fused step kernel."""
    bx, rows, pipe = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().lb_get_launch(ctypes.c_void_p(h), ctypes.byref(bx), ctypes.byref(rows),
                                ctypes.byref(pipe)), "lb_get_launch")
    return bx.value, rows.value, pipe.value


def lb_set_launch(h: int, block_x: int, rows_per_cta: int, pipeline: int) -> None:
    _check(load().lb_set_launch(ctypes.c_void_p(h), int(block_x), int(rows_per_cta),
                                int(pipeline)), "lb_set_launch")


def lb_set_wait_limit(h: int, cycles: int, test_skip_copies: int = 0) -> None:
    _check(load().lb_set_wait_limit(ctypes.c_void_p(h), int(cycles), int(test_skip_copies)),
           "lb_set_wait_limit")


def lb_energy_noalloc(psi, rho, nx: int, ny: int, G1: float, G2: float, out=None,
                      stream: int = 0):
    """(E_s, E_m, E_bulk, mass) of device fields psi and rho without any device
    allocation (scratch in a static device array; see include/lb.h). With
    out=None the result comes back through a host buffer."""
    host = out is None
    if host:
        out = np.zeros(4)
    st = load().lb_energy_noalloc(_ptr(psi), _ptr(rho), int(nx), int(ny), float(G1), float(G2),
                                  _ptr(out), ctypes.c_void_p(stream or None))
    _check(st, "lb_energy_noalloc")
    return tuple(float(v) for v in out) if host else out


def lb_check_guards(h: int) -> int:
    """Number of the state's device buffers whose guard regions were overwritten."""
    n = ctypes.c_int(0)
    _check(load().lb_check_guards(ctypes.c_void_p(h), ctypes.byref(n)), "lb_check_guards")
    return n.value


def lb_debug_fail_alloc(after: int) -> None:
    load().lb_debug_fail_alloc(int(after))


def lb_debug_damage_guard(h: int, buffer: int) -> None:
    _check(load().lb_debug_damage_guard(ctypes.c_void_p(h), int(buffer)), "lb_debug_damage_guard")


def lb_state_bytes(h: int) -> int:
    return int(load().lb_state_bytes(ctypes.c_void_p(h)))


def lb_save_state(h: int, dst=None):
    """Save the state into dst (a uint8 array/tensor of lb_state_bytes) or a new NumPy buffer."""
    n = lb_state_bytes(h)
    if dst is None:
        dst = np.empty(n, dtype=np.uint8)
    _check(load().lb_save_state(ctypes.c_void_p(h), _ptr(dst), n), "lb_save_state")
    return dst


def lb_load_state(h: int, src) -> None:
    nbytes = src.nbytes if hasattr(src, "nbytes") else src.numel() * src.element_size()
    _check(load().lb_load_state(ctypes.c_void_p(h), _ptr(src), int(nbytes)), "lb_load_state")


def lb_adjoint(h: int, steps: int, rho_target, checkpoint_every: int = 0, grad_rho=None):
    """(J, grad_rho, (dJ/dG1, dJ/dG2)) for a fresh FP32 state; grad_rho may be a
    caller array/tensor (host or device) or None for a new NumPy array."""
    if isinstance(rho_target, np.ndarray):
        rho_target = np.ascontiguousarray(rho_target, dtype=np.float64)
    J = ctypes.c_double(0.0)
    gG = (ctypes.c_double * 2)()
    out = grad_rho
    if out is None:
        shape = getattr(rho_target, "shape", None)
        out = np.empty(shape if shape is not None else (0,))
    _check(load().lb_adjoint(ctypes.c_void_p(h), int(steps), _ptr(rho_target),
                             int(checkpoint_every), ctypes.byref(J), _ptr(out), gG),
           "lb_adjoint")
    return float(J.value), out, (float(gG[0]), float(gG[1]))


def lb_objective(h: int, rho_target) -> float:
    """J = E_s + E_m + sum (rho - rho_target)^2 of the current state (FP64 sums on the
    device; for FP32 states the same kernel and order as lb_adjoint's J)."""
    if isinstance(rho_target, np.ndarray):
        rho_target = np.ascontiguousarray(rho_target, dtype=np.float64)
    J = ctypes.c_double(0.0)
    _check(load().lb_objective(ctypes.c_void_p(h), _ptr(rho_target), ctypes.byref(J)),
           "lb_objective")
    return float(J.value)


def lb_batch_init(params_list, rho_list, stream: int = 0) -> int:
    """Handle of a batch of len(params_list) replicas; rho_list[r] is [ny_r, nx_r] float64."""
    n = len(params_list)
    if n != len(rho_list):
        raise ValueError("one initial density per parameter set")
    P = (lb_params * n)(*params_list)
    keep = [np.ascontiguousarray(r, dtype=np.float64) if isinstance(r, np.ndarray) else r
            for r in rho_list]
    ptrs = (ctypes.c_void_p * n)(*[_ptr(r) for r in keep])
    h = ctypes.c_void_p()
    _check(load().lb_batch_init(ctypes.byref(h), n, P, ptrs, ctypes.c_void_p(stream or None)),
           "lb_batch_init")
    return h.value


def lb_batch_step(h: int, n: int) -> None:
    _check(load().lb_batch_step(ctypes.c_void_p(h), int(n)), "lb_batch_step")


def lb_batch_energy(h: int, replica: int):
    out = (ctypes.c_double * 4)()
    _check(load().lb_batch_energy(ctypes.c_void_p(h), int(replica), out), "lb_batch_energy")
    return tuple(out)


def lb_batch_fields(h: int, replica: int, rho=None, ux=None, uy=None) -> None:
    _check(load().lb_batch_fields(ctypes.c_void_p(h), int(replica), _ptr(rho), _ptr(ux),
                                  _ptr(uy)), "lb_batch_fields")


def lb_batch_trace(h: int, replica: int, cap: int = 65536) -> np.ndarray:
    buf = np.zeros((max(cap, 1), 5))
    cnt = ctypes.c_int(0)
    _check(load().lb_batch_trace(ctypes.c_void_p(h), int(replica),
                                 buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(cap),
                                 ctypes.byref(cnt)), "lb_batch_trace")
    return buf[: cnt.value].copy()


def lb_batch_get_launch(h: int):
    bx, rows, g = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().lb_batch_get_launch(ctypes.c_void_p(h), ctypes.byref(bx), ctypes.byref(rows),
                                      ctypes.byref(g)), "lb_batch_get_launch")
    return bx.value, rows.value, g.value


def lb_batch_set_launch(h: int, block_x: int, rows_per_cta: int, use_graph: int = 1) -> None:
    _check(load().lb_batch_set_launch(ctypes.c_void_p(h), int(block_x), int(rows_per_cta),
                                      int(use_graph)), "lb_batch_set_launch")


def lb_batch_check_guards(h: int) -> int:
    n = ctypes.c_int(0)
    _check(load().lb_batch_check_guards(ctypes.c_void_p(h), ctypes.byref(n)),
           "lb_batch_check_guards")
    return n.value


def lb_batch_count(h) -> int:
    return int(load().lb_batch_count(ctypes.c_void_p(h)))


def lb_batch_time(h) -> int:
    return int(load().lb_batch_time(ctypes.c_void_p(h)))


def lb_batch_destroy(h) -> None:
    load().lb_batch_destroy(ctypes.c_void_p(h))


def lb_time(h) -> int:
    return int(load().lb_time(ctypes.c_void_p(h)))


def lb_destroy(h) -> None:
    load().lb_destroy(ctypes.c_void_p(h))
