"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (no GPU).  The planted copies are compiled to a
temporary directory; the oracle itself is never modified."""
import os
import subprocess

import pytest

import pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "lbm_oracle.c")

# (name, exact text in the oracle, planted replacement)
MUTATIONS = [
    ("eq15_last_term_without_eps", "- 3.0 / eps * uF", "- 3.0 * uF"),
    ("eq15_wrong_prefactor", "(1.0 - 1.0 / (2.0 * tau))", "(1.0 - 1.0 / tau)"),
    ("eq15_dropped_cross_term", "+ 9.0 / eps * eu * eF", "+ 0.0 * eu * eF"),
    ("eq14_sign_of_u2", "- 3.0 / (2.0 * eps) * uu", "+ 3.0 / (2.0 * eps) * uu"),
    ("eq14_missing_eps", "9.0 / (2.0 * eps) * eu * eu", "9.0 / 2.0 * eu * eu"),
    ("eq17_no_half_force", "ux = (mx + 0.5 * rho * eps * p->Gx) / den;", "ux = mx / den;"),
    ("eq17_darcy_without_eps", "double den = rho + 0.5 * (eps * nu / ka) * rho;",
     "double den = rho + 0.5 * (nu / ka) * rho;"),
    ("eq8_sign_of_drag", "Fx = -(eps * nu / ka) * ux + eps * p->Gx;",
     "Fx = (eps * nu / ka) * ux + eps * p->Gx;"),
    ("quadratic_wrong_power", "c1 * vmag);", "c1 * vmag * vmag);"),
    ("eq2_forchheimer_dropped", "- (eps * Feps * sqrt(inv_k)) * umag * ux +", "+"),
    ("viscosity", "(p->tau - 0.5) / 3.0 / p->J", "(p->tau - 0.5) / 6.0 / p->J"),
    ("eq12_relaxation", "fpost[i] = f[i] - (f[i] - feq[i]) / p->tau + Fi[i];",
     "fpost[i] = f[i] - (f[i] - feq[i]) * p->tau + Fi[i];"),
    ("eq13_transposed_diagonal", "{0, 0, 1, 0, -1, 1, 1, -1, -1}", "{0, 0, 1, 0, -1, 1, -1, -1, 1}"),
    ("weights", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}", "1.0 / 36.0, 1.0 / 36.0, 1.0 / 9.0}"),
    ("eq7_exponent_sign", "pow(kn, -0.4348)", "pow(kn, 0.4348)"),
    ("eq6_slip_sign", "const double b = -1.0;", "const double b = 1.0;"),
    ("eq7_constant", "1.358 / (1.0 + 0.170", "1.358 / (1.0 + 1.70"),
    ("eq3_not_applied", "return k_i * orc_fc(kn);", "return k_i;"),
    ("bounce_back_same_direction", "s->f[j * 9 + i] = s->fs[j * 9 + opp];",
     "s->f[j * 9 + i] = s->fs[j * 9 + i];"),
    ("pressure_density_not_imposed", "orc_feq(rho_b, u_n, eps_b, feq_b);",
     "orc_feq(rho_n, u_n, eps_b, feq_b);"),
    ("pressure_gradient_without_eps", "/ 3.0 / eps_mean;", "/ 3.0;"),
    ("impermeable_force", "Fx = -2.0 * mx / rho;", "Fx = 0.0;"),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(orc, source, tmp_path, name, old, new):
    assert source.count(old) == 1, f"mutation anchor for {name} not unique/found"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(src), "-lm"], check=True)
    caught = None
    with orc.use_library(str(so)):
        for pin in pins.ALL_PINS:
            try:
                pin(orc)
            except Exception as exc:  # AssertionError, non-convergence, NaN
                caught = (pin.__name__, type(exc).__name__)
                break
    assert caught is not None, f"planted mistake {name} passed every pin"
