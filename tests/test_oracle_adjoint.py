"""Pins of the oracle's reverse-mode gradient.

J = E_s(T) + E_m(T) + sum_x (rho(x, T) - rho*(x))^2 (Sec. 5 energy plus a misfit
to a seeded target). The gradient with respect to the initial density field,
G1 and G2 is checked against central finite differences of J (h = 1e-4, FP64),
and one reverse step against the transpose identity <M v, w> = <v, M^T w> with
M v taken by central differences of one forward step — neither check looks
inside the reverse code."""
import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import inputs

H = 1e-4


def _case(n=24, seed=11):
    r0 = inputs.noisy_density(n, n, seed, mean=0.7, amp=0.05)
    tgt = inputs.noisy_density(n, n, seed + 1, mean=0.7, amp=0.05)
    return r0, tgt


@pytest.mark.parametrize("G2,omega,steps", [(0.0, 1.0, 30), (0.5, 1.0, 40), (0.3, 1.3, 25)])
def test_gradient_matches_central_differences(G2, omega, steps):
    r0, tgt = _case()
    kw = dict(G1=-5.0, G2=G2, omega=omega)
    J, g, gG = oracle.gradient(r0, tgt, steps, **kw)
    assert J == pytest.approx(oracle.objective(r0, tgt, steps, **kw)[0], rel=1e-14)
    rng = np.random.default_rng(3)
    for _ in range(2):
        v = rng.standard_normal(r0.shape)
        fd = (oracle.objective(r0 + H * v, tgt, steps, **kw)[0] -
              oracle.objective(r0 - H * v, tgt, steps, **kw)[0]) / (2 * H)
        assert abs((g * v).sum() - fd) <= 1e-6 * abs(fd)
    # a single site (the field gradient is local, not just its projections)
    e = np.zeros_like(r0)
    e[5, 7] = 1.0
    fd = (oracle.objective(r0 + H * e, tgt, steps, **kw)[0] -
          oracle.objective(r0 - H * e, tgt, steps, **kw)[0]) / (2 * H)
    assert abs(g[5, 7] - fd) <= 1e-6 * abs(fd) + 1e-9
    for k, name in enumerate(("G1", "G2")):
        kp, km = dict(kw), dict(kw)
        kp[name] += H
        km[name] -= H
        fd = (oracle.objective(r0, tgt, steps, **kp)[0] -
              oracle.objective(r0, tgt, steps, **km)[0]) / (2 * H)
        assert abs(gG[k] - fd) <= 1e-6 * abs(fd)


def test_reverse_step_is_the_transpose_of_the_step():
    r0, _ = _case(n=17, seed=5)
    rng = np.random.default_rng(9)
    f = oracle.step(oracle.init(r0), G1=-5.0, G2=0.6)     # a non-equilibrium state
    v = rng.standard_normal(f.shape)
    w = rng.standard_normal(f.shape)
    eps = 1e-6
    Mv = (oracle.step(f + eps * v, G1=-5.0, G2=0.6, omega=1.2) -
          oracle.step(f - eps * v, G1=-5.0, G2=0.6, omega=1.2)) / (2 * eps)
    lam, gG = oracle.adjoint_step(f, w, G1=-5.0, G2=0.6, omega=1.2)
    lhs, rhs = (Mv * w).sum(), (v * lam).sum()
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)
    # the explicit G terms: a larger difference step (the quantity is small, so the
    # round-off of the quotient, not its truncation, limits a 1e-6 step)
    for k, name in enumerate(("G1", "G2")):
        kp = dict(G1=-5.0, G2=0.6, omega=1.2)
        km = dict(kp)
        kp[name] += H
        km[name] -= H
        d = ((oracle.step(f, **kp) - oracle.step(f, **km)) / (2 * H) * w).sum()
        assert abs(gG[k] - d) <= 1e-6 * abs(d)


def test_terminal_gradient_of_energy_alone():
    """T = 0: dJ/drho_init is psi' dE/dpsi + 2 (rho - rho*) exactly (no steps)."""
    r0, tgt = _case(n=12, seed=21)
    J, g, gG = oracle.gradient(r0, tgt, 0, G1=-5.0, G2=0.4)
    rng = np.random.default_rng(1)
    v = rng.standard_normal(r0.shape)
    fd = (oracle.objective(r0 + H * v, tgt, 0, G1=-5.0, G2=0.4)[0] -
          oracle.objective(r0 - H * v, tgt, 0, G1=-5.0, G2=0.4)[0]) / (2 * H)
    assert abs((g * v).sum() - fd) <= 1e-7 * abs(fd)
