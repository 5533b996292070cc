"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests retypes the oracle's formulas: each checks it against a
printed number (tests/golden/), a closed form, an invariant, an independent
formulation (Fourier symbol, linearised 9x9 mode matrix, 40-digit brute
force), or a special case that reduces to the textbook single-belt model.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1008_2865_gb300 import inputs


def _vectors(e):
    """All integer lattice vectors with |c|^2 == e inside the 5x5 stencil."""
    return [(x, y) for y in range(-2, 3) for x in range(-2, 3) if x * x + y * y == e]


def _exact(v, maxden=20000):
    return Fraction(v).limit_denominator(maxden)


def _links(table1, d2q9, G1, G2):
    """[(cx, cy, K_c)] with K_c = G1 w_c + G2 p_c built from the golden tables."""
    w = {e: wv for e, n, wv in d2q9}
    p = {e: pv for b, e, n, pv in table1}
    out = []
    for e in (1, 2, 4, 5, 8):
        for c in _vectors(e):
            out.append((c[0], c[1], G1 * float(w.get(e, 0)) + G2 * float(p[e])))
    return out


def _symbol(links, k):
    """S(k) = sum_c K_c c sin(k.c): the force's Fourier symbol (vector)."""
    s = np.zeros(2)
    for cx, cy, K in links:
        s += K * np.array([cx, cy]) * math.sin(k[0] * cx + k[1] * cy)
    return s


# --------------------------------------------------------------------------- Table 1
def test_link_table_matches_table1(table1, d2q9):
    cx, cy, w, p = oracle.link_table()
    e = cx.astype(int) ** 2 + cy.astype(int) ** 2
    assert e[0] == 0
    speeds = {(int(a), int(b)) for a, b in zip(cx[1:], cy[1:])}
    assert len(speeds) == 24 and (0, 0) not in speeds
    assert speeds == {c for ee in (1, 2, 4, 5, 8) for c in _vectors(ee)}
    for belt, ee, n, pv in table1:
        sel = np.nonzero(e == ee)[0]
        assert len(sel) == n
        for k in sel:
            assert _exact(p[k]) == pv, (ee, p[k], pv)
            assert p[k] == float(pv)
    wmap = {ee: wv for ee, n, wv in d2q9}
    for k in range(25):
        assert _exact(w[k]) == wmap.get(int(e[k]), Fraction(0))
    # belt 1 = the eight D2Q9 speeds in indices 1..8, belt 2 = the rest
    assert set(e[1:9]) == {1, 2} and set(e[9:]) == {4, 5, 8}


def test_weight_normalisations_eq_weights_1_2(constants):
    """Eq. weights_1 and weights_2, and the 12/7 fourth-moment ratio of Eq. gamma."""
    cx, cy, w, p = oracle.link_table()
    P = [_exact(v) for v in p]
    Wt = [_exact(v) for v in w]
    cs2 = Fraction(constants["cs2"])
    assert sum(Wt) == 1
    assert sum(P) == 1                              # includes the rest weight p_s0
    assert P[0] == Fraction(247, 420)               # rest weight left by Eq. weights_1
    assert abs(p[0] - 247 / 420) <= 2e-16
    x2 = [int(a) ** 2 for a in cx]
    y2 = [int(b) ** 2 for b in cy]
    assert sum(pp * a for pp, a in zip(P, x2)) == cs2   # per Cartesian component
    assert sum(pp * b for pp, b in zip(P, y2)) == cs2
    assert sum(ww * a for ww, a in zip(Wt, x2)) == cs2
    m4p = sum(pp * a * a for pp, a in zip(P, x2))
    m4w = sum(ww * a * a for ww, a in zip(Wt, x2))
    assert m4p / m4w == Fraction(constants["gamma_coefficient_G2"])


# --------------------------------------------------------------------------- psi
def test_psi_is_correctly_rounded_sc_form():
    """psi = sqrt(rho0)(1 - exp(-rho/rho0)) (Sec. 2) with exp correctly rounded."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 300
    rho = np.random.default_rng(7).uniform(0.01, 4.0, 3000)
    got = oracle.psi(rho)
    for r, g in zip(rho, got):
        e = float(mpmath.exp(-mpmath.mpf(float(r))))
        assert g == 1.0 - e
    # rho0 != 1: sqrt(rho0) scale and rho/rho0
    got2 = oracle.psi(rho, rho0=2.0)
    ref2 = math.sqrt(2.0) * (1.0 - np.array([float(mpmath.exp(-mpmath.mpf(float(r)) / 2)) for r in rho]))
    assert np.max(np.abs(got2 - ref2)) <= 4e-16


# --------------------------------------------------------------------------- force
def _plane_wave_symbol(G1, G2, m, L):
    """Extract S(k) from the oracle's force on psi = a + b cos(k.x)."""
    y, x = np.mgrid[0:L, 0:L]
    k = 2 * np.pi * np.array(m, float) / L
    ph = k[0] * x + k[1] * y
    a, b = 0.5, 1e-3
    fx, fy = oracle.force(a + b * np.cos(ph), G1, G2)
    s = np.sin(ph)
    # F = b S(k) sin(k.x) (a + b cos(k.x)); the b^2 part is orthogonal to sin(k.x)
    return np.array([(fx * s).sum(), (fy * s).sum()]) * 2 / (L * L) / (a * b), k


@pytest.mark.parametrize("G1,G2", [(-5.0, 0.0), (-5.0, 0.6), (0.0, 1.0), (-4.9, 15.1)])
def test_force_matches_fourier_symbol(table1, d2q9, G1, G2):
    """The oracle's force on a plane wave equals the exact lattice symbol (sign included)."""
    links = _links(table1, d2q9, G1, G2)
    for m in [(1, 0), (3, 4), (7, 2)]:
        s, k = _plane_wave_symbol(G1, G2, m, 64)
        ref = _symbol(links, k)
        assert np.allclose(s, ref, rtol=1e-9, atol=1e-13), (m, s, ref)


def test_force_taylor_coefficients_eq_ftot(constants):
    """Small-k expansion of the force = Eq. ftot with A1 = G1+G2 and 12/7 (Eq. gamma).

    Along x, F = -psi [cs2 A1 d_x psi + cs2^2/2 (G1 + 12/7 G2) d_x lap psi] + O(k^5),
    i.e. S(k)/k = cs2 A1 - cs2^2/2 (G1 + 12/7 G2) k^2 + O(k^4).
    """
    cs2 = float(Fraction(constants["cs2"]))
    lam = float(Fraction(constants["gamma_coefficient_G2"]))
    c1 = float(Fraction(constants["ftot_gradient_coefficient"]))
    c2 = float(Fraction(constants["ftot_laplacian_coefficient"]))
    L = 1024
    for G1, G2 in [(-5.0, 0.0), (-5.0, 0.6), (-4.9, 4.0)]:
        ks, ss = [], []
        for mm in (1, 2, 3, 4, 5, 6):
            # a 1D wave is enough: use an L x 5 lattice with psi constant in y
            x = np.arange(L)
            k = 2 * np.pi * mm / L
            a, b = 0.5, 1e-3
            ps = (a + b * np.cos(k * x))[None, :].repeat(5, 0)
            fx, _ = oracle.force(ps, G1, G2)
            s = (fx[2] * np.sin(k * x)).sum() * 2 / L / (a * b)
            ks.append(k)
            ss.append(s / k)
        ks = np.array(ks)
        A = np.stack([np.ones_like(ks), ks ** 2, ks ** 4], 1)
        coef = np.linalg.lstsq(A, np.array(ss), rcond=None)[0]
        A1 = G1 + G2
        assert abs(coef[0] - c1 * cs2 * A1) <= 1e-9 * abs(A1)
        assert abs(coef[1] + c2 * cs2 ** 2 * (G1 + lam * G2)) <= 1e-6 * (abs(G1) + abs(G2))


def test_force_eighth_order_isotropy(constants):
    """Sec. 3: the E(8) set is isotropic to 8th order, the D2Q9 set only to 4th.

    k = 2pi/L (5, 0) and 2pi/L (3, 4) have the same length; an isotropic symbol
    gives the same magnitude and no transverse part for both.
    """
    assert int(constants["isotropy_order"]) == 8
    L = 512

    def aniso(G1, G2):
        s1, k1 = _plane_wave_symbol(G1, G2, (5, 0), L)
        s2, k2 = _plane_wave_symbol(G1, G2, (3, 4), L)
        n2 = np.linalg.norm(k2)
        par = s2 @ k2 / n2
        perp = (s2[0] * k2[1] - s2[1] * k2[0]) / n2
        return max(abs(s1[0] - par), abs(perp), abs(s1[1])) / abs(s1[0])

    assert aniso(0.0, 1.0) < 1e-11       # p weights alone: isotropic through O(k^8)
    assert aniso(1.0, 0.0) > 1e-8        # D2Q9 weights: anisotropic at O(k^4)


def test_single_belt_reduces_to_eq_forza(d2q9):
    """G2 = 0: Eq. FORCE is the textbook force F = -G psi sum_i w_i psi(x+c_i) c_i."""
    rng = np.random.default_rng(3)
    ps = rng.uniform(0.2, 0.8, (9, 11))
    G = -4.7
    fx, fy = oracle.force(ps, G, 0.0)
    rx = np.zeros_like(ps)
    ry = np.zeros_like(ps)
    wmap = {e: float(wv) for e, n, wv in d2q9}
    for cx in (-1, 0, 1):
        for cy in (-1, 0, 1):
            if cx == cy == 0:
                continue
            nb = np.roll(ps, (-cy, -cx), (0, 1))        # psi(x + c)
            rx += wmap[cx * cx + cy * cy] * nb * cx
            ry += wmap[cx * cx + cy * cy] * nb * cy
    np.testing.assert_allclose(fx, -G * ps * rx, rtol=0, atol=1e-15)
    np.testing.assert_allclose(fy, -G * ps * ry, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- invariants
def test_uniform_state_stays_uniform():
    rho0 = np.full((12, 9), 0.7)
    rho, ux, uy, _ = oracle.run(rho0, 60, G1=-5.0, G2=0.6)
    assert np.max(np.abs(rho - 0.7)) <= 1e-14
    assert np.max(np.abs(ux)) <= 1e-15 and np.max(np.abs(uy)) <= 1e-15


@pytest.mark.parametrize("G2,omega", [(0.0, 1.0), (0.6, 1.0), (0.3, 1.4)])
def test_mass_and_momentum_conservation(G2, omega):
    """Collision conserves mass, streaming permutes; sum_x F = 0 keeps total momentum 0."""
    rho0 = inputs.noisy_density(40, 33, seed=5, amp=0.05)
    rho, ux, uy, tr = oracle.run(rho0, 300, omega=omega, G1=-5.0, G2=G2, trace_every=10)
    m0 = rho0.sum()
    assert abs(rho.sum() - m0) <= 1e-13 * m0
    assert np.max(np.abs(tr[:, 1] - m0)) <= 1e-13 * m0
    # physical check that the run did something
    assert rho.max() - rho.min() > 0.1
    # total momentum sum rho u: j* = j + F per site and sum_x F = 0
    assert abs((rho * ux).sum()) <= 1e-11 and abs((rho * uy).sum()) <= 1e-11


def test_translation_is_exact():
    rho0 = inputs.noisy_density(20, 17, seed=9, amp=0.02)
    a = oracle.run(rho0, 40, G1=-5.0, G2=0.5)
    b = oracle.run(np.roll(rho0, (3, -5), (0, 1)), 40, G1=-5.0, G2=0.5)
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(np.roll(u, (3, -5), (0, 1)), v)


def test_d4_symmetry():
    """Mirror x, mirror y and transpose map solutions onto solutions (rounding aside)."""
    rho0 = inputs.noisy_density(24, 24, seed=4, amp=0.02)
    kw = dict(G1=-5.0, G2=0.5)
    r, ux, uy, _ = oracle.run(rho0, 30, **kw)
    r2, ux2, uy2, _ = oracle.run(rho0[:, ::-1], 30, **kw)          # x -> -x
    assert np.allclose(r2, r[:, ::-1], rtol=0, atol=1e-12)
    assert np.allclose(ux2, -ux[:, ::-1], rtol=0, atol=1e-12)
    assert np.allclose(uy2, uy[:, ::-1], rtol=0, atol=1e-12)
    r3, ux3, uy3, _ = oracle.run(rho0.T, 30, **kw)                  # x <-> y
    assert np.allclose(r3, r.T, rtol=0, atol=1e-12)
    assert np.allclose(ux3, uy.T, rtol=0, atol=1e-12)
    assert np.allclose(uy3, ux.T, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------- energies
@pytest.mark.parametrize("G1,G2", [(-5.0, 0.0), (-5.0, 0.6), (-4.9, 9.8)])
def test_energy_uniform_closed_form(G1, G2, table1):
    """Sec. 5: for uniform psi, E_s + E_m = E_bulk = A1/2 N psi^2 (Eq. Ebulk) exactly,
    with E_m = G2/2 N psi^2 sum_m p and E_s carrying the rest of the weight."""
    ny, nx = 7, 9
    psi = 0.6
    es, em, eb = oracle.energy(np.full((ny, nx), psi), G1, G2)
    N = nx * ny
    pm = sum(n * pv for b, e, n, pv in table1 if b == "m")
    assert pm == Fraction(596, 15120)
    assert math.isclose(eb, (G1 + G2) / 2 * N * psi * psi, rel_tol=1e-14)
    assert math.isclose(es + em, eb, rel_tol=1e-13, abs_tol=1e-13)
    assert math.isclose(em, G2 / 2 * N * psi * psi * float(pm), rel_tol=1e-13, abs_tol=1e-15)
    assert math.isclose(es, N * psi * psi / 2 * (G1 + G2 * float(1 - pm)), rel_tol=1e-13)


def test_energy_weak_gradient_expansion():
    """Next order of the Sec. 5 expansion: sum_c K_c psi(x+c) = A1 psi + A1/6 lap psi + ...,
    so E - E_bulk -> -(A1/12) sum |grad psi|^2 for a smooth field (summation by parts)."""
    L = 256
    y, x = np.mgrid[0:L, 0:L]
    k = 2 * np.pi / L
    psi = 0.5 + 0.05 * np.cos(k * x) + 0.03 * np.sin(2 * k * y)
    for G1, G2 in [(-5.0, 0.0), (-5.0, 0.8)]:
        es, em, eb = oracle.energy(psi, G1, G2)
        A1 = G1 + G2
        grad2 = (0.05 * k * np.sin(k * x)) ** 2 + (0.06 * k * np.cos(2 * k * y)) ** 2
        pred = -(A1 / 12.0) * grad2.sum()
        assert math.isclose(es + em - eb, pred, rel_tol=2e-3)


# --------------------------------------------------------------------------- linear theory
def _d2q9_list(d2q9):
    w = {e: float(wv) for e, n, wv in d2q9}
    return [(cx, cy, w[cx * cx + cy * cy]) for cy in (-1, 0, 1) for cx in (-1, 0, 1)]


def _mode_matrix(pops, links, k, rho_bar, omega, rho0=1.0):
    """Linearised one-step map of a Fourier mode e^{ik.x} about (rho_bar, u = 0):
    collision C (Eq. 4 at the shifted velocity u + F/(omega rho), force linearised
    through psi' = exp(-rho/rho0)/sqrt(rho0)), then streaming diag(e^{-ik.c_i})."""
    psib = math.sqrt(rho0) * (1 - math.exp(-rho_bar / rho0))
    dpsi = math.exp(-rho_bar / rho0) / math.sqrt(rho0)
    S = _symbol(links, k)
    q = len(pops)
    C = np.zeros((q, q), complex)
    for i, (cxi, cyi, wi) in enumerate(pops):
        for j, (cxj, cyj, _) in enumerate(pops):
            C[i, j] = omega * wi * (1 + 3 * (cxi * cxj + cyi * cyj))
            C[i, j] += -3j * wi * psib * dpsi * (cxi * S[0] + cyi * S[1])
        C[i, i] += 1 - omega
    D = np.diag([np.exp(-1j * (k[0] * cx + k[1] * cy)) for cx, cy, _ in pops])
    return D @ C


@pytest.mark.parametrize("G1,G2,omega,m", [(-5.0, 0.0, 1.0, (1, 0)), (-5.0, 0.6, 1.0, (2, 1)),
                                           (-3.0, 0.4, 1.3, (3, 3)), (-5.0, 0.9, 0.8, (5, 2))])
def test_linear_mode_growth(table1, d2q9, G1, G2, omega, m):
    """A small Fourier mode evolves as the 9x9 linearised mode matrix says."""
    L, n, eps, rho_bar = 32, 25, 1e-6, 0.7
    pops = _d2q9_list(d2q9)
    links = _links(table1, d2q9, G1, G2)
    k = 2 * np.pi * np.array(m) / L
    y, x = np.mgrid[0:L, 0:L]
    ph = k[0] * x + k[1] * y
    rho, _, _, _ = oracle.run(rho_bar + eps * np.cos(ph), n, omega=omega, G1=G1, G2=G2)
    meas = (rho * np.exp(-1j * ph)).sum() / (L * L)
    M = _mode_matrix(pops, links, k, rho_bar, omega)
    a = np.array([wi * eps / 2 for _, _, wi in pops], complex)
    pred = (np.linalg.matrix_power(M, n) @ a).sum()
    assert abs(meas - pred) <= 1e-6 * abs(pred) + 1e-17, (meas, pred)


def test_critical_point(table1, d2q9, constants):
    """Sec. 2: G_cr = -4 at rho_cr = rho0 ln 2. The linearised long-wave growth
    factor crosses 1 there, and the oracle's small noise decays above and grows below."""
    assert float(constants["G_cr"]) == -4.0
    rho_cr = math.log(2.0)
    pops = _d2q9_list(d2q9)
    k = np.array([2 * np.pi / 256, 0.0])

    def growth(G):
        M = _mode_matrix(pops, _links(table1, d2q9, G, 0.0), k, rho_cr, 1.0)
        return max(abs(np.linalg.eigvals(M)))

    assert growth(-3.98) < 1.0 < growth(-4.02)
    # the oracle: noise about rho_cr decays for G = -3.6, grows for G = -4.4
    rho0 = rho_cr + 1e-4 * (2 * inputs.uniform(11, 64 * 64).reshape(64, 64) - 1)
    amp = []
    for G in (-3.6, -4.4):
        r, _, _, _ = oracle.run(rho0, 600, G1=G, G2=0.0)
        amp.append(np.std(r))
    s0 = np.std(rho0)
    assert amp[0] < 0.5 * s0 and amp[1] > 10 * s0


# --------------------------------------------------------------------------- interface
@pytest.mark.parametrize("G2,liq,gas,tol", [(0.0, 1.93, 0.156, 1e-6), (0.5, 1.49, 0.253, 2e-5)])
def test_flat_interface_pressure_balance(G2, liq, gas, tol):
    """A flat liquid slab relaxes to bulk densities with equal pressure
    p = rho + A1 psi^2 / 2 (the EOS of Sec. 3 in units of cs2), and rho_g < ln 2 < rho_l.

    On the lattice the balance is exact in a steady state: summed across an
    interface the force telescopes to -(A1/6)(psi_l^2 - psi_g^2), which the
    momentum flux cs2 (rho_l - rho_g) must cancel."""
    nx, ny = 64, 5
    x = np.arange(nx) + 0.5
    prof = gas + (liq - gas) * 0.5 * (np.tanh((x - 16) / 3) - np.tanh((x - 48) / 3))
    rho, _, _, _ = oracle.run(prof[None, :].repeat(ny, 0), 20000, G1=-5.0, G2=G2)
    A1 = -5.0 + G2
    rl, rg = rho[2, 32], rho[2, 0]

    def p(r):
        s = 1 - math.exp(-r)
        return r + A1 * s * s / 2

    assert rg < math.log(2) < rl
    assert abs(p(rl) - p(rg)) <= tol * abs(p(rl))


# --------------------------------------------------------------------------- brute force
def test_brute_force_step_5x5(table1, d2q9):
    """One step on a 5x5 periodic lattice redone in 40-digit arithmetic, push form,
    force summed per |c|^2 class with K_c = G1 w + G2 p from the golden tables."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 40
    n = 5
    G1, G2, omega, rho0 = -5.0, 0.7, 1.2, 1.0
    rng = np.random.default_rng(12)
    pops = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    wmap = {e: wv for e, nn, wv in d2q9}
    pmap = {e: pv for b, e, nn, pv in table1}
    f = np.empty((9, n, n))
    for i, (cx, cy) in enumerate(pops):
        f[i] = float(wmap[cx * cx + cy * cy]) * rng.uniform(0.5, 1.0, (n, n)) + 0.01 * rng.uniform(-1, 1, (n, n))
    got = oracle.step(f, omega=omega, G1=G1, G2=G2, rho0=rho0)

    F = [[[mp.mpf(float(f[i, y, x])) for x in range(n)] for y in range(n)] for i in range(9)]
    rho = [[sum(F[i][y][x] for i in range(9)) for x in range(n)] for y in range(n)]
    psi = [[mp.sqrt(rho0) * (1 - mp.exp(-rho[y][x] / rho0)) for x in range(n)] for y in range(n)]
    K = {}
    for e in (1, 2, 4, 5, 8):
        wv = wmap.get(e, Fraction(0))
        K[e] = mp.mpf(G1) * mp.mpf(wv.numerator) / wv.denominator + \
            mp.mpf(G2) * mp.mpf(pmap[e].numerator) / pmap[e].denominator
    out = [[[None] * n for _ in range(n)] for _ in range(9)]
    for y in range(n):
        for x in range(n):
            fx = fy = mp.mpf(0)
            for e in (1, 2, 4, 5, 8):
                for cx, cy in _vectors(e):
                    nb = psi[(y + cy) % n][(x + cx) % n]
                    fx += K[e] * nb * cx
                    fy += K[e] * nb * cy
            fx, fy = -psi[y][x] * fx, -psi[y][x] * fy
            jx = sum(F[i][y][x] * pops[i][0] for i in range(9))
            jy = sum(F[i][y][x] * pops[i][1] for i in range(9))
            r = rho[y][x]
            vx = (jx + fx / omega) / r
            vy = (jy + fy / omega) / r
            for i, (cx, cy) in enumerate(pops):
                wv = wmap[cx * cx + cy * cy]
                cu = cx * vx + cy * vy
                feq = mp.mpf(wv.numerator) / wv.denominator * r * \
                    (1 + 3 * cu + mp.mpf(9) / 2 * cu * cu - mp.mpf(3) / 2 * (vx * vx + vy * vy))
                out[i][(y + cy) % n][(x + cx) % n] = F[i][y][x] - omega * (F[i][y][x] - feq)
    ref = np.array([[[float(out[i][y][x]) for x in range(n)] for y in range(n)] for i in range(9)])
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 1e-14
