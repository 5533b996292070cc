"""The oracle's pins must catch plausible mistakes.

Each case compiles a copy of the oracle source with one planted error (a sign,
a dropped term, a wrong weight, a transposed operand, a reversed index) and
runs the pin tests against that copy; at least one pin must fail. The
planted errors live only in temporary copies on the CPU.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "lbsc_oracle.c")).read()

MUTANTS = {
    "force sign": [("*Fx = -(Fsx + Fmx);", "*Fx = (Fsx + Fmx);"),
                   ("*Fy = -(Fsy + Fmy);", "*Fy = (Fsy + Fmy);")],
    "G2 dropped on belt 1": [(" + P->G2 * ps * sx;", ";"), (" + P->G2 * ps * sy;", ";")],
    "belt-2 weight p(5)": [("2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0,\n",
                            "2.0 / 945.0, 2.0 / 945.0, 2.0 / 945.0, 1.0 / 945.0,\n")],
    "belt-2 speed transposed": [("mx += PM[k] * pn * MCX[k];", "mx += PM[k] * pn * MCY[k];")],
    "streaming reversed": [("f_out[i * N + site(P, x + CX[i], y + CY[i])] = fs;",
                            "f_out[i * N + site(P, x - CX[i], y - CY[i])] = fs;")],
    "velocity shift without omega": [("const double orho = om * rho;", "const double orho = rho;")],
    "equilibrium 2nd-order coefficient": [("4.5 * cu * cu", "3.0 * cu * cu")],
    "relaxation sign": [("fi - om * (fi - feq)", "fi - om * (feq - fi)")],
    "momentum component": [("ay += CY[i] * fi;", "ay += CX[i] * fi;")],
    "psi scale rho0": [("exp_cr(-rho / rho0)", "exp_cr(-rho * rho0)")],
    "energy rest term": [("double ss = (P->G1 * W[0] + P->G2 * p0) * ps;", "double ss = 0.0 * ps;")],
    "energy belt-2 coupling": [("sm += P->G2 * PM[k]", "sm += P->G1 * PM[k]")],
    "energy half factor": [("em += 0.5 * ps * sm;", "em += ps * sm;")],
    "adjoint: velocity term of the collision": [("rb -= (vbx * vx + vby * vy) / r;",
                                                 "rb += (vbx * vx + vby * vy) / r;")],
    "adjoint: force transpose gather dropped": [("pb += K * (CX[i] * Qx[n] + CY[i] * Qy[n]);",
                                                 "pb += 0.0 * K;")],
    "adjoint: reverse streaming direction": [("ls[i] = lam_next[i * N + site(P, x + CX[i], y + CY[i])];",
                                              "ls[i] = lam_next[i * N + site(P, x - CX[i], y - CY[i])];")],
    "adjoint: energy derivative factor": [("E += 0.5 * ps * sk;", "E += 0.5 * ps * sk + 0.0;"),
                                          ("dEdpsi[y * nx + x] = sk;", "dEdpsi[y * nx + x] = 0.5 * sk;")],
    "diagonal weight": [("1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};",
                         "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 35.0};")],
}


def _fixtures():
    from conftest import read_golden
    from fractions import Fraction
    table1 = [(b, int(e), int(n), Fraction(p)) for b, e, n, p in read_golden("table1_weights.txt")]
    d2q9 = [(int(e), int(n), Fraction(w)) for e, n, w in read_golden("d2q9_weights.txt")]
    constants = {r[0]: r[1] for r in read_golden("paper_constants.txt")}
    return table1, d2q9, constants


def _pin_calls(table1, d2q9, constants):
    """The pin tests, with their fixtures and a representative parameter set each."""
    yield lambda: pins.test_link_table_matches_table1(table1, d2q9)
    yield lambda: pins.test_weight_normalisations_eq_weights_1_2(constants)
    yield lambda: pins.test_psi_is_correctly_rounded_sc_form()
    for G1, G2 in [(-5.0, 0.6), (0.0, 1.0)]:
        yield lambda G1=G1, G2=G2: pins.test_force_matches_fourier_symbol(table1, d2q9, G1, G2)
    yield lambda: pins.test_single_belt_reduces_to_eq_forza(d2q9)
    yield lambda: pins.test_uniform_state_stays_uniform()
    yield lambda: pins.test_mass_and_momentum_conservation(0.3, 1.4)
    yield lambda: pins.test_translation_is_exact()
    for G1, G2 in [(-5.0, 0.6), (-4.9, 9.8)]:
        yield lambda G1=G1, G2=G2: pins.test_energy_uniform_closed_form(G1, G2, table1)
    for args in [(-5.0, 0.6, 1.0, (2, 1)), (-3.0, 0.4, 1.3, (3, 3))]:
        yield lambda args=args: pins.test_linear_mode_growth(table1, d2q9, *args)
    yield lambda: pins.test_brute_force_step_5x5(table1, d2q9)
    import test_oracle_adjoint as adj
    yield lambda: adj.test_reverse_step_is_the_transpose_of_the_step()
    yield lambda: adj.test_gradient_matches_central_differences(0.5, 1.0, 10)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    src = SRC
    for old, new in MUTANTS[name]:
        assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new)
    lib = oracle.compile_source(src, str(tmp_path / "liblbsc_oracle_mutant.so"))
    table1, d2q9, constants = _fixtures()
    caught = []
    with oracle.use_library(lib):
        for call in _pin_calls(table1, d2q9, constants):
            try:
                call()
            except AssertionError:
                caught.append(call)
                break
    assert caught, f"no pin failed for the planted mistake: {name}"


def test_unmutated_source_passes_all_pins(tmp_path):
    lib = oracle.compile_source(SRC, str(tmp_path / "liblbsc_oracle_copy.so"))
    table1, d2q9, constants = _fixtures()
    with oracle.use_library(lib):
        for call in _pin_calls(table1, d2q9, constants):
            call()
