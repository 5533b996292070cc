"""GPU adjoint: lb_adjoint (FP32 state and adjoint, FP64 gradient accumulation)
against the FP64 oracle's reverse sweep, which is itself pinned to central
finite differences (tests/test_oracle_adjoint.py).

J = E_s(T) + E_m(T) + sum (rho(T) - rho*)^2 on a separate periodic 64 x 64
lattice (the "64x64 crop" of the 512^2 adjoint workload), G1 = -5, G2 = 0.5,
rho_init and rho* seeded as the +-1% noise about 0.7 (seeds 11 and 12).
Bars: J to 1e-6, the G1/G2 gradients to 1e-4 and the field gradient to 1e-4 in
relative 2-norm — the FP32 forward trajectory and the FP32 adjoint stay within
about 1e-5 of FP64 over these horizons, well inside the bars."""
import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import LBError, Lattice, capi, inputs

pytestmark = pytest.mark.gpu


def _case(n=64):
    r0 = inputs.noisy_density(n, n, 11, mean=0.7, amp=0.01, mode="rel")
    tgt = inputs.noisy_density(n, n, 12, mean=0.7, amp=0.01, mode="rel")
    return r0, tgt


@pytest.mark.parametrize("G2,omega,steps", [(0.5, 1.0, 60), (0.0, 1.0, 100), (0.3, 1.3, 40)])
def test_adjoint_matches_oracle(G2, omega, steps):
    r0, tgt = _case()
    Jo, go, gGo = oracle.gradient(r0, tgt, steps, omega=omega, G1=-5.0, G2=G2)
    with Lattice(r0, omega=omega, G1=-5.0, G2=G2, trace_every=0) as lat:
        J, g, gG = lat.adjoint(steps, tgt)
        assert lat.t == steps
    assert abs(J - Jo) <= 1e-6 * abs(Jo)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    for k in range(2):
        assert abs(gG[k] - gGo[k]) <= 1e-4 * abs(gGo[k])


def test_adjoint_matches_oracle_at_the_full_horizon():
    """The 512^2 adjoint workload's horizon, T = 2000, on its 64 x 64 periodic
    stand-in (G1 = -5, G2 = 0.5, seeds 11 and 12): the FP32 forward and adjoint stay
    on the FP64 trajectory closely enough that J and dJ/dG1, dJ/dG2 agree with the
    oracle's reverse sweep to better than 1e-6 (measured 5.9e-7, 5.8e-7, 5.8e-7)
    and the field gradient to 1.1e-4 in relative 2-norm. Bars: J 2e-6, dJ/dG 1e-5,
    field gradient 3e-4 (about 3x the measured error)."""
    r0, tgt = _case()
    Jo, go, gGo = oracle.gradient(r0, tgt, 2000, G1=-5.0, G2=0.5)
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        J, g, gG = lat.adjoint(2000, tgt)
    assert abs(J - Jo) <= 2e-6 * abs(Jo)
    for k in range(2):
        assert abs(gG[k] - gGo[k]) <= 1e-5 * abs(gGo[k])
    assert np.linalg.norm(g - go) <= 3e-4 * np.linalg.norm(go)


def _J_gpu(r0, tgt, steps, prec, G1=-5.0, G2=0.5):
    with Lattice(r0, G1=G1, G2=G2, prec=prec, trace_every=0) as lat:
        lat.step(steps)
        return lat.objective(tgt)


@pytest.mark.parametrize("steps", [20, 100, 300])
def test_adjoint_against_gpu_central_differences(steps):
    """dJ/dG1, dJ/dG2 and a directional derivative along a seeded field direction v
    from the FP32 adjoint against central differences (h = 1e-4) of J evaluated by
    the library itself (lb_objective, FP64 sums) on FP64 states, which follow the
    oracle's trajectory bit for bit. Measured agreement of the G derivatives:
    1e-8 (T = 20), 1e-6 (T = 100, 300); bar 2e-5. The direction v has random signs,
    so <grad J, v> is a small sum of cancelling terms; its error is measured on the
    scale |grad J| |v| that bounds it (Cauchy-Schwarz): the FP32 field gradient is
    within 1e-5 of the FP64 one in relative 2-norm up to T = 300; bar 1e-5 |grad J|
    |v|. The field step is h_v = 1e-6: by T = 300 the unstable modes have grown so
    that the O(h^2) error of h = 1e-4 along v is 3% of the derivative, while FP64
    rounding of J (about 1e-12) stays far below h_v |grad J| |v|."""
    r0, tgt = _case()
    h = 1e-4
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        _, g, gG = lat.adjoint(steps, tgt)
    d1 = (_J_gpu(r0, tgt, steps, "fp64", G1=-5.0 + h) -
          _J_gpu(r0, tgt, steps, "fp64", G1=-5.0 - h)) / (2 * h)
    d2 = (_J_gpu(r0, tgt, steps, "fp64", G2=0.5 + h) -
          _J_gpu(r0, tgt, steps, "fp64", G2=0.5 - h)) / (2 * h)
    assert abs(d1 - gG[0]) <= 2e-5 * abs(gG[0])
    assert abs(d2 - gG[1]) <= 2e-5 * abs(gG[1])
    v = inputs.noisy_density(64, 64, 13, mean=0.0, amp=1.0, mode="abs")
    hv = 1e-6
    dv = (_J_gpu(r0 + hv * v, tgt, steps, "fp64") -
          _J_gpu(r0 - hv * v, tgt, steps, "fp64")) / (2 * hv)
    assert abs(dv - float(np.sum(g * v))) <= 1e-5 * np.linalg.norm(g) * np.linalg.norm(v)


def test_adjoint_against_fp32_central_differences():
    """The same check with J evaluated on FP32 states (the adjoint's own forward
    arithmetic), h = 1e-4, at T = 20: the FP32 rounding of the two perturbed
    trajectories puts about 5e-4 of noise into the difference quotient (measured
    4.7e-4 and 4.5e-4 for G1 and G2); bar 1e-3."""
    r0, tgt = _case()
    h = 1e-4
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        _, _, gG = lat.adjoint(20, tgt)
    d1 = (_J_gpu(r0, tgt, 20, "fp32", G1=-5.0 + h) - _J_gpu(r0, tgt, 20, "fp32", G1=-5.0 - h)) / (2 * h)
    d2 = (_J_gpu(r0, tgt, 20, "fp32", G2=0.5 + h) - _J_gpu(r0, tgt, 20, "fp32", G2=0.5 - h)) / (2 * h)
    assert abs(d1 - gG[0]) <= 1e-3 * abs(gG[0])
    assert abs(d2 - gG[1]) <= 1e-3 * abs(gG[1])


def test_adjoint_is_independent_of_checkpoint_spacing():
    r0, tgt = _case(48)
    res = []
    for C in (0, 1, 7, 30):
        with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
            res.append(lat.adjoint(30, tgt, checkpoint_every=C))
    for J, g, gG in res[1:]:
        assert J == res[0][0] and gG == res[0][2] and np.array_equal(g, res[0][1])


def test_adjoint_forward_equals_plain_run_and_device_output():
    torch = pytest.importorskip("torch")
    r0, tgt = _case(96)
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=10) as lat:
        grad = torch.empty((96, 96), dtype=torch.float64, device="cuda")
        J, _, gG = lat.adjoint(50, torch.from_numpy(tgt).cuda(), grad_rho=grad)
        rho_a, _, _ = lat.fields()
        tr_a = lat.trace()
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=10) as lat:
        lat.step(50)
        rho_b, _, _ = lat.fields()
        tr_b = lat.trace()
        J2, g2, gG2 = (None, None, None)
    assert np.array_equal(rho_a, rho_b) and np.array_equal(tr_a, tr_b)
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        J2, g2, gG2 = lat.adjoint(50, tgt)
    assert J == J2 and gG == gG2 and np.array_equal(grad.cpu().numpy(), g2)


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_1008_2865_gb300.autograd import LBObjective
    r0, tgt = _case(40)
    rho = torch.from_numpy(r0).cuda().requires_grad_(True)
    G1 = torch.tensor(-5.0, dtype=torch.float64, requires_grad=True)
    G2 = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    J = LBObjective.apply(rho, G1, G2, torch.from_numpy(tgt).cuda(), 25)
    (2.0 * J).backward()
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        Jr, gr, gGr = lat.adjoint(25, tgt)
    assert float(J) == Jr
    assert np.array_equal(rho.grad.cpu().numpy(), 2.0 * gr)
    assert float(G1.grad) == 2.0 * gGr[0] and float(G2.grad) == 2.0 * gGr[1]
    # without gradients the forward evaluates J with lb_objective (the adjoint's own
    # terminal kernel): the same J bit for bit
    with torch.no_grad():
        J0 = LBObjective.apply(rho.detach(), G1.detach(), G2.detach(),
                               torch.from_numpy(tgt).cuda(), 25)
    assert float(J0) == Jr


def test_adjoint_arguments():
    r0, tgt = _case(16)
    with Lattice(r0, prec="fp64") as lat:
        with pytest.raises(LBError) as ei:
            lat.adjoint(5, tgt)
        assert ei.value.status == capi.LB_ERR_STATE
    with Lattice(r0) as lat:
        lat.step(1)
        with pytest.raises(LBError) as ei:
            lat.adjoint(5, tgt)
        assert ei.value.status == capi.LB_ERR_STATE


def test_objective_equals_adjoint_J_and_oracle():
    """lb_objective after T steps gives the adjoint's J bit for bit (same terminal
    kernel and order) for host and device targets; on an FP64 state, whose
    trajectory is the oracle's bit for bit, it matches the oracle's J (Sec. 5
    energy plus misfit) to 1e-12."""
    torch = pytest.importorskip("torch")
    r0, tgt = _case(64)
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        J, _, _ = lat.adjoint(40, tgt)
    with Lattice(r0, G1=-5.0, G2=0.5, trace_every=0) as lat:
        lat.step(40)
        assert lat.objective(tgt) == J
        assert lat.objective(torch.from_numpy(tgt).cuda()) == J
    Jo, _ = oracle.objective(r0, tgt, 40, G1=-5.0, G2=0.5)
    with Lattice(r0, prec="fp64", G1=-5.0, G2=0.5, trace_every=0) as lat:
        lat.step(40)
        J64 = lat.objective(tgt)
    assert abs(J64 - Jo) <= 1e-12 * abs(Jo)
    with Lattice(r0, prec="fp16_delta", G1=-5.0, G2=0.5, trace_every=0) as lat:
        lat.step(40)
        J16 = lat.objective(tgt)
    assert abs(J16 - Jo) <= 1e-3 * abs(Jo)
