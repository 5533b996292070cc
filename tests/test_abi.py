"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol include/lb.h declares, and argument validation needs no GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1008_2865_gb300 import build as lbbuild
from paper_1008_2865_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    lbbuild.build()
    return capi.load()


def test_header_declares_the_boundary():
    names = _declared("lb.h")
    for n in ("lb_init", "lb_step", "lb_energy", "lb_fields", "lb_trace", "lb_time", "lb_destroy",
              "lb_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lbbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lb_[a-z_0-9]+)\b", out))
    for header in os.listdir(os.path.join(ROOT, "include")):
        for name in _declared(header):
            assert name in exported, f"{name} declared in {header} but not exported"
            assert hasattr(lib, name)


def _prototypes(header):
    """{name: number of parameters} of the functions a header declares."""
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(lb_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_header(lib):
    """Every function the binding declares passes as many arguments as the C prototype."""
    protos = {}
    for header in os.listdir(os.path.join(ROOT, "include")):
        protos.update(_prototypes(header))
    assert len(protos) >= 20
    for name, nargs in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, f"{name} has no argtypes in the binding"
        assert len(fn.argtypes) == nargs, (name, len(fn.argtypes), nargs)


def test_params_struct_layout_matches_header(lib):
    # the ctypes mirror must match the C layout: offsets of doubles after ints
    P = capi.lb_params
    assert ctypes.sizeof(P) == 72
    assert P.omega.offset == 8 and P.rho_ref.offset == 56 and P.device.offset == 64


def test_status_strings(lib):
    for st in (0, -1, -2, -3, -4, -5, -6):
        assert capi.lb_status_str(st)
    assert capi.lb_status_str(17) == "unknown status"


@pytest.mark.parametrize("bad", [dict(nx=4), dict(ny=3), dict(omega=0.0), dict(omega=2.0),
                                 dict(G1=float("nan")), dict(G2=float("inf")), dict(rho0=0.0),
                                 dict(trace_every=-1), dict(prec=7), dict(psi_form=3),
                                 dict(rho_ref=float("nan")), dict(device=-1),
                                 dict(nx=20000, ny=20000), dict(nx=15456, ny=15456),
                                 dict(nx=33, ny=4_000_000)])
def test_invalid_parameters_rejected_on_host(lib, bad):
    kw = dict(nx=16, ny=16)
    kw.update(bad)
    psi_form = kw.pop("psi_form", 0)
    p = capi.make_params(**kw, psi_form=psi_form)
    rho = np.full((max(kw["ny"], 1), max(kw["nx"], 1)) if kw["nx"] * kw["ny"] < 1e7 else (1, 1), 0.7)
    h = ctypes.c_void_p(123)
    st = lib.lb_init(ctypes.byref(h), ctypes.byref(p), rho.ctypes.data, None)
    assert st == capi.LB_ERR_ARG
    assert h.value is None


def test_null_arguments(lib):
    assert lib.lb_init(None, None, None, None) == capi.LB_ERR_ARG
    assert lib.lb_step(None, 1) == capi.LB_ERR_ARG
    assert lib.lb_energy(None, None) == capi.LB_ERR_ARG
    assert lib.lb_fields(None, None, None, None) == capi.LB_ERR_ARG
    assert lib.lb_trace(None, None, 0, None) == capi.LB_ERR_ARG
    assert lib.lb_time(None) == -1
    lib.lb_destroy(None)


def test_product_path_does_not_use_the_oracle():
    """The package and bench's GPU arm never import the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_1008_2865_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lbsc_oracle" not in text, f
