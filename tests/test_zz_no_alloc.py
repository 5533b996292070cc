"""lb_energy_noalloc: the pseudo-energy / mass reduction for callers that
cannot allocate device memory (for example code whose device memory all comes
from a framework's own pool). Its scratch is a static device array inside the
library; this file checks that two calls in a row through the C ABI agree
with lb_energy on the same state, and that sizes beyond the array's capacity
are refused. The file is named to be collected last."""
import math

import numpy as np
import pytest

from paper_1008_2865_gb300 import LBError, Lattice, capi, inputs

pytestmark = pytest.mark.gpu


def _psi(torch, rho, rho0=1.0):
    return math.sqrt(rho0) * (1.0 - torch.exp(-rho / rho0))


# one CTA covers 16,384 sites: 96 x 80 and 131 x 67 are one partial CTA, 512 x 512 is
# 16 full CTAs, 1000 x 999 is 61 CTAs with a partial last one, 4096 x 4096 is 1024 CTAs
@pytest.mark.parametrize("nx,ny,G2", [(96, 80, 0.5), (131, 67, 0.0), (512, 512, 0.9),
                                      (1000, 999, 0.6), (4096, 4096, 0.3)])
def test_noalloc_energy_matches_lb_energy_twice(nx, ny, G2):
    torch = pytest.importorskip("torch")
    rho0 = inputs.noisy_density(nx, ny, seed=21, mean=0.7, amp=0.05)
    with Lattice(rho0, prec="fp64", G1=-5.0, G2=G2, trace_every=0) as lat:
        lat.step(30 if nx * ny <= 1 << 20 else 3)
        ref = lat.energy()
        rho = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        lat.fields(rho=rho)
    psi = _psi(torch, rho)
    torch.cuda.synchronize()
    first = capi.lb_energy_noalloc(psi, rho, nx, ny, -5.0, G2)
    second = capi.lb_energy_noalloc(psi, rho, nx, ny, -5.0, G2)
    assert first == second
    for got in (first, second):
        for g, r in zip(got, ref):
            if r == 0.0:
                assert abs(g) <= 1e-12
            else:
                assert abs(g - r) <= 1e-12 * abs(r)
    # device output, read after the stream is done
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    capi.lb_energy_noalloc(psi, rho, nx, ny, -5.0, G2, out=out,
                           stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert tuple(out.cpu().numpy()) == first


def test_noalloc_rejects_sizes_beyond_its_scratch_and_host_fields():
    torch = pytest.importorskip("torch")
    small = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(LBError) as ei:
        capi.lb_energy_noalloc(small, small, 16384, 8193, -5.0, 0.0)
    assert ei.value.status == capi.LB_ERR_ARG
    with pytest.raises(LBError) as ei:
        capi.lb_energy_noalloc(small, small, 4, 8, -5.0, 0.0)
    assert ei.value.status == capi.LB_ERR_ARG
    host = np.ones((8, 8))
    with pytest.raises(LBError) as ei:
        capi.lb_energy_noalloc(host, host, 8, 8, -5.0, 0.0)
    assert ei.value.status == capi.LB_ERR_ARG


def test_noalloc_refuses_host_result_during_capture():
    """A host result needs a stream synchronisation, which a capture forbids: the call
    is refused with LB_ERR_ARG before anything is enqueued, and the capture goes on."""
    torch = pytest.importorskip("torch")
    rho = torch.full((16, 16), 0.7, dtype=torch.float64, device="cuda")
    psi = _psi(torch, rho)
    side = torch.cuda.Stream()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            with pytest.raises(LBError) as ei:
                capi.lb_energy_noalloc(psi, rho, 16, 16, -5.0, 0.0, stream=side.cuda_stream)
            x.add_(1.0)
    assert ei.value.status == capi.LB_ERR_ARG
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0


def test_noalloc_refuses_fields_of_another_device():
    """psi/rho in memory of a device other than the current one are refused before any
    launch (needs two visible GPUs)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    other = torch.ones((8, 8), dtype=torch.float64, device="cuda:1")
    with torch.cuda.device(0):
        with pytest.raises(LBError) as ei:
            capi.lb_energy_noalloc(other, other, 8, 8, -5.0, 0.0)
    assert ei.value.status == capi.LB_ERR_ARG
