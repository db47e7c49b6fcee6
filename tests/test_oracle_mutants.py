"""Sensitivity of the oracle's pins: plant one plausible mistake at a time in a copy of
the oracle (on the CPU), rebuild it, and check that at least one pin in
``test_oracle_pins.py`` fails.  Each mutant names the passage of the paper it breaks."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "asx_oracle.c")

# name: (passage, original text, mutated text)
MUTANTS = {
    "flux_without_projection": ("given mass flux reading (l q n_side . n)",
                                "const double qin = l * q * (ns1 * n1 + ns2 * n2);", "const double qin = l * q;"),
    "flux_without_momentum": ("given mass flux reading (inflow momentum)", "J1 += qin * uin * (-ns1);",
                              "J1 += 0.0 * uin;"),
    "dirichlet_pressure_sign": ("Eq. numerics-bc ghost through Eq. fvm_2D_eq_frac.01",
                                "S1 -= 0.5 * l * dw * hat * n1;\n                        S2 -= 0.5 * l * dw * hat * n2;\n                        out_rate += l * thh * vn;",
                                "S1 += 0.5 * l * dw * hat * n1;\n                        S2 += 0.5 * l * dw * hat * n2;\n                        out_rate += l * thh * vn;"),
    "thacker_no_linear_resistance": ("Eq. eq_soil_friction_thacker (tau h v)",
                                     "orc_friction(m_new + dt * p->tau * h_new, beta",
                                     "orc_friction(m_new, beta"),
    "visc_sign": ("Eq. eq_visc1 (v_j - v_i)", "J2 += l * cij * mu * (v2[j] - v2[i]);",
                  "J2 += l * cij * mu * (v2[i] - v2[j]);"),
    "visc_min_speed": ("Eq. eq_visc1 (c_(i,j) = max)", "const double cij = ci > cj ? ci : cj;",
                       "const double cij = ci < cj ? ci : cj;"),
    "visc_arithmetic_mean": ("Eq. eq_visc1 (harmonic mean mu)",
                             "const double mu = den > 0.0 ? 2.0 * m[i] * m[j] / den : 0.0;",
                             "const double mu = 0.5 * den;"),
    "visc_without_edge_length": ("Eq. eq_artif_visc (l_(i,j))", "J2 += l * cij * mu * (v2[j] - v2[i]);",
                                 "J2 += cij * mu * (v2[j] - v2[i]);"),
    "pressure_sign": ("Eq. fvm_2D_eq_frac.01 (S)", "S1 -= 0.5 * l * dw * hat * n1;", "S1 += 0.5 * l * dw * hat * n1;"),
    "pressure_half": ("Eq. fvm_2D_eq_frac.01 (S, factor 1/2)",
                      "S1 -= 0.5 * l * dw * hat * n1;\n                    S2 -= 0.5 * l * dw * hat * n2;",
                      "S1 -= l * dw * hat * n1;\n                    S2 -= l * dw * hat * n2;"),
    "downwind": ("Eq. fvm_2D_eq.06 (upwind)",
                 "if (vn > 0.0) thh = m[i];\n                    else if (vn < 0.0) thh = m[j];",
                 "if (vn > 0.0) thh = m[j];\n                    else if (vn < 0.0) thh = m[i];"),
    "hat_reversed": ("Eq. fvm_2D_eq.05 (tie rule)", "hat = (dw < 0.0) ? m[i] : m[j];", "hat = (dw < 0.0) ? m[j] : m[i];"),
    "rain_times_theta": ("Eq. fvm_2D_eq_frac.07 (source M)", "double m_new = m_star + dt * rain;",
                         "double m_new = m_star + dt * rain * p->theta[i];"),
    "rain_left_end": ("Eq. fvm_2D_eq_frac.07 (M at t^{n+1})", "const double rain = orc_rain_rate(p, t_next);",
                      "const double rain = orc_rain_rate(p, t_next - dt);"),
    "odd_row_offset": ("Sec. 2.2 (a) (neighbours)", "case 1: rr = r + 1; cc = odd ? c + 1 : c; break;",
                       "case 1: rr = r + 1; cc = odd ? c : c + 1; break;"),
    "normal_sign": ("Sec. 2.2 (a) (outward normal)", "static const int sg[6] = {0, 1, 1, 0, -1, -1};",
                    "static const int sg[6] = {0, 1, 1, 0, 1, -1};"),
    "K_without_1_minus_theta": ("Eq. eq_K_h_theta",
                                "return p->alpha_p[i] * h * (1.0 - p->theta[i]) + p->theta[i] * p->alpha_s[i];",
                                "return p->alpha_p[i] * h + p->theta[i] * p->alpha_s[i];"),
    "K_without_theta_soil": ("Eq. eq_K_h_theta",
                             "return p->alpha_p[i] * h * (1.0 - p->theta[i]) + p->theta[i] * p->alpha_s[i];",
                             "return p->alpha_p[i] * h * (1.0 - p->theta[i]) + p->alpha_s[i];"),
    "no_momentum_flux": ("Eq. fvm_2D_eq_frac.01 (J)", "J1 -= l * thh * vb1 * vn;", ";"),
    "momentum_flux_cell_velocity": ("Eq. fvm_2D_eq.04", "J1 -= l * thh * vb1 * vn;", "J1 -= l * thh * v1[i] * vn;"),
    "momentum_without_inertia": ("Eq. fvm_2D_eq_frac.05-2",
                                 "const double g1 = m[i] * v1[i] + dt / sigma * (J1 + S1);",
                                 "const double g1 = dt / sigma * (J1 + S1);"),
    "friction_old_depth": ("Eq. fvm_2D_eq_frac.06-2 (K at h^{n+1})", "h_new = m_new / p->theta[i];", "h_new = hi;"),
    "mu_factor": ("Eq. miu-formula", "double den = alpha + sqrt(alpha * alpha + 4.0 * beta * ng);",
                  "double den = alpha + sqrt(alpha * alpha + 2.0 * beta * ng);"),
    "depth_without_theta": ("Eq. eq_gforce (w uses h, not theta h)", "const double hj = m[j] / p->theta[j];",
                            "const double hj = m[j];"),
    "phi_five_sides": ("Eq. fvm_2D_eq_frac.13", "return orc_sigma(l) / (6.0 * l);", "return orc_sigma(l) / (5.0 * l);"),
    "wave_speed": ("Eq. fvm_2D_eq_frac.13 (c_i)",
                   "double c = sqrt(v1[i] * v1[i] + v2[i] * v2[i]) + sqrt(p->g * h);",
                   "double c = sqrt(v1[i] * v1[i] + v2[i] * v2[i]) + p->g * h;"),
    "free_side_inflow": ("free discharge reading (outflow only)",
                         "if (vn > 0.0) {\n                            L -= l * m[i] * vn;",
                         "if (vn != 0.0) {\n                            L -= l * m[i] * vn;"),
    "outflow_misbooked": ("ledger (Table table_BasinSusita identity)", "out_rate += l * m[i] * vn;",
                          "out_rate += 0.5 * l * m[i] * vn;"),
    "cell_area_apothem": ("hexagon area with l = circumradius",
                          "double orc_sigma(double l) { return 1.5 * sqrt(3.0) * l * l; }",
                          "double orc_sigma(double l) { return 2.0 * sqrt(3.0) * l * l; }"),
    "interface_velocity_sum": ("Eq. fvm_2D_eq.04", "const double vb2 = (v2[i] + v2[j]) / 2.0;",
                               "const double vb2 = (v2[i] + v2[j]);"),
    "potential_without_g": ("Eq. eq_gforce", "const double dw = g * ((p->z[j] - p->z[i]) + (hj - hi));",
                            "const double dw = ((p->z[j] - p->z[i]) + (hj - hi));"),
}


@pytest.fixture(scope="module")
def mutant_dir():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, mutant_dir):
    passage, before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(before, after, 1)
    c = os.path.join(mutant_dir, name + ".c")
    so = os.path.join(mutant_dir, name + ".so")
    with open(c, "w") as f:
        f.write(mutated)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", so, c, "-lm"])
    env = dict(os.environ, ASX_ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-q", "-x", "-p", "no:cacheprovider"], env=env, capture_output=True, text=True,
                       cwd=ROOT, timeout=600)
    assert r.returncode != 0, f"no pin caught the mutant '{name}' ({passage}):\n{r.stdout[-2000:]}"
