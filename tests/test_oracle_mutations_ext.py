"""Planted mistakes in the oracle's physical inputs (Eq. 9-11), first-order
factor (Eq. 4-5), dynamic Knudsen number, velocity histogram (Fig. 6),
central-difference gradient, steady-state residual and mass: each must be
caught by the pins written for that function (no GPU).  The planted copies are compiled to a temporary
directory; the oracle itself is never modified."""
import os
import subprocess

import pytest

import test_oracle_gradient as grad
import test_oracle_histogram as hist
import test_oracle_physical as phys
import test_oracle_reductions as red

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "lbm_oracle.c")

PHYS = [lambda: phys.test_kozeny_carman_is_kozeny_form(0.3, 40e-9),
        lambda: phys.test_herd_radius_is_capillary_bundle(1e-18, 0.2),
        lambda: phys.test_mean_free_path_kinetic_form(1000.0, 323.0),
        phys.test_first_order_factor]
DYN = [lambda: phys.test_dynamic_kn_darcy_closed_form(0),
       lambda: phys.test_dynamic_kn_darcy_closed_form(1),
       phys.test_dynamic_kn_zero_beta_is_static]
HIST = [hist.test_uniform_flow_fills_last_bin, hist.test_no_flow_fills_first_bin,
        hist.test_channel_histogram_follows_eq20, hist.test_layered_darcy_flow_bins]
GRAD = [lambda: grad.test_uniform_sum_matches_scalar_recurrence(0),
        lambda: grad.test_uniform_sum_matches_scalar_recurrence(1), grad.test_node_indexing]
RES = red.RESIDUAL_PINS
MASS = red.MASS_PINS

# (name, exact text in the oracle, planted replacement, pins that must catch it)
MUTATIONS = [
    ("eq9_constant", "const double C = d * d / 180.0;", "const double C = d * d / 150.0;", PHYS),
    ("eq9_exponent", "return C * eps * eps * eps / ((1.0 - eps) * (1.0 - eps));",
     "return C * eps * eps / ((1.0 - eps) * (1.0 - eps));", PHYS),
    ("eq11_constant", "return 8.886e-2 * sqrt(k_mD / eps) * 1e-6;",
     "return 8.886e-3 * sqrt(k_mD / eps) * 1e-6;", PHYS),
    ("eq11_darcy_unit", "const double k_mD = k_d / 9.869e-16;", "const double k_mD = k_d / 9.869e-13;",
     PHYS),
    ("eq10_missing_pi", "return mu / p * sqrt(3.14159265358979323846 * R * T / (2.0 * M));",
     "return mu / p * sqrt(R * T / (2.0 * M));", PHYS),
    ("eq5_factor", "double orc_fc_first_order(double kn) { return 1.0 + 4.0 * kn; }",
     "double orc_fc_first_order(double kn) { return 1.0 + 3.0 * kn; }", PHYS),
    ("dynamic_kn_inverted", "return s->ki[j] * orc_fc_model(s->kn[j] / q, p->kn_model);",
     "return s->ki[j] * orc_fc_model(s->kn[j] * q, p->kn_model);", DYN),
    ("dynamic_kn_ignored", "  if (p->kn_beta == 0.0) return s->ka[j];",
     "  if (1) return s->ka[j];", DYN),
    ("dynamic_kn_wrong_density", "  const double q = 1.0 + p->kn_beta * (rho - p->rho0);",
     "  const double q = 1.0 + p->kn_beta * (rho - 1.0 - p->rho0);", DYN),
    ("histogram_rounds", "k = (int)floor(speed[j] / mx * nbins);",
     "k = (int)floor(speed[j] / mx * nbins + 0.5);", HIST),
    ("histogram_drops_last", "if (k > nbins - 1) k = nbins - 1;", "if (k > nbins - 1) continue;",
     HIST),
    ("fd_one_sided", "out[m] = (kg[2 * m] - kg[2 * m + 1]) / (2.0 * h);",
     "out[m] = (kg[2 * m] - kg[2 * m + 1]) / h;", GRAD),
    ("fd_linear_in_k", "pk[j] = k_i[j] * exp(sign * h);", "pk[j] = k_i[j] + sign * h;", GRAD),
    ("fd_wrong_node", "const int64_t j = nodes[e / 2];", "const int64_t j = nodes[e / 2] + 1;",
     GRAD),
    ("residual_no_sqrt", "return sqrt(num) / sqrt(den);", "return num / den;", RES),
    ("residual_norm_of_snapshot", "den += u[0] * u[0] + u[1] * u[1];",
     "den += ux_prev[j] * ux_prev[j] + uy_prev[j] * uy_prev[j];", RES),
    ("residual_drops_y", "num += dx * dx + dy * dy;", "num += dx * dx;", RES),
    ("residual_over_plate_rows",
     "double num = 0.0, den = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n"
     "    if (orc_is_wall_row(p, y)) continue;",
     "double num = 0.0, den = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n", RES),
    ("residual_skips_last_column", "  double num = 0.0, den = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n"
     "    if (orc_is_wall_row(p, y)) continue;\n    for (int x = 0; x < p->nx; ++x) {",
     "  double num = 0.0, den = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n"
     "    if (orc_is_wall_row(p, y)) continue;\n    for (int x = 0; x < p->nx - 1; ++x) {", RES),
    ("mass_over_plate_rows",
     "double m = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n    if (orc_is_wall_row(p, y)) continue;",
     "double m = 0.0;\n  for (int y = 0; y < p->ny; ++y) {\n", MASS),
    ("mass_drops_rest_population", "for (int i = 0; i < 9; ++i) m += s->f[j * 9 + i];",
     "for (int i = 1; i < 9; ++i) m += s->f[j * 9 + i];", MASS),
]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name,old,new,checks", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(orc, source, tmp_path, name, old, new, checks):
    assert source.count(old) == 1, f"mutation anchor for {name} not unique/found"
    src = tmp_path / "mutant.c"
    src.write_text(source.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-o", str(so), str(src), "-lm"], check=True)
    caught = None
    with orc.use_library(str(so)):
        for check in checks:
            try:
                check()
            except Exception as exc:  # AssertionError, ValueError, non-convergence, NaN
                caught = type(exc).__name__
                break
    assert caught is not None, f"planted mistake {name} passed every pin"
