"""Planted mistakes: each entry below changes one line of a copy of the oracle the way a
slip in writing it from the paper could (a dropped term, a wrong sign, index or coefficient,
a transposed operand, a mistyped table entry), and the test checks that the oracle's pins
(tests/test_oracle_*.py) reject that copy.  The copy is built in a temporary directory and
handed to the pins through LBM_ORACLE_UNDER_TEST (read by the `orc` fixture of conftest.py);
the oracle itself is never modified.  Each entry names the pin file expected to reject it
first, so a pin that loses its power shows up here.

One kind of planted slip is known to pass every pin and is therefore not listed: the
advection speed of the convective outflow, for the flow and the temperature populations alike
(reading 19 of the design notes; the blend (old + U inner) / (1 + U) with U replaced by 1, or
the inner value taken alone).  Every steady state is a fixed point of the blend for any U, and the
pins (the exact uniform stream, the flux balance of the walled channel) are steady; the speed
shapes only the transient, for which the paper gives nothing to compare with.  Nor is the
corner convention of node walls (a corner site takes the velocity of its lowest-numbered wall
face, reading 26): the paper leaves it open, and no pin has two differently moving walls
meeting at a corner.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file in oracle/, text, planted replacement, what the slip is, pin file, pin test)
MUTANTS = [
    ("feq_porosity_dropped", "lbm_oracle.c",
     "eu * eu / (2.0 * phi * CS2 * CS2)", "eu * eu / (2.0 * CS2 * CS2)",
     "Eq. 24: the 1/phi of the quadratic term",
     "test_oracle_lattice.py", "feq_moments"),
    ("stilde_coefficient", "lbm_oracle.c",
     "S[1] = 38.0 * rho0 * uF / phi;", "S[1] = 19.0 * rho0 * uF / phi;",
     "Eq. 23: the energy-moment coefficient",
     "test_oracle_lattice.py", "stilde"),
    ("source_half_factor_dropped", "lbm_oracle.c",
     "(1.0 - 0.5 * L->s[k]) * S[k]", "S[k]",
     "Eq. 9: the (I - Lambda/2) factor of the source",
     "test_oracle_collision.py", "post_collision_momentum"),
    ("transform_transposed", "lbm_oracle.c",
     "m[k] += D->m[k * q + i] * f[i];", "m[k] += D->m[i * q + k] * f[i];",
     "m = M f with M transposed",
     "test_oracle_collision.py", "fixed_point"),
    ("half_force_dropped", "lbm_oracle.c",
     "v[a] = s / rho0 + 0.5 * phi * G[a];", "v[a] = s / rho0 + phi * G[a];",
     "Eq. 28: the half-step force in v",
     "test_oracle_lattice.py", "velocity_solves_eq26"),
    ("l0_factor", "lbm_oracle.c",
     "double l0 = 0.5 * (1.0 + phi * 0.5 * nu / K);", "double l0 = 0.5 * (1.0 + phi * nu / K);",
     "Eq. 28: the 1/2 in l0",
     "test_oracle_lattice.py", "velocity_solves_eq26"),
    ("forchheimer_sqrt_k", "lbm_oracle.c",
     "(phi * Fphi / sqrt(K)) * umag * u[a]", "(phi * Fphi / K) * umag * u[a]",
     "Eq. 4: sqrt(K) of the Forchheimer term",
     "test_oracle_lattice.py", "velocity_solves_eq26"),
    ("buoyancy_reference_dropped", "lbm_oracle.c",
     "G[a] = L->buoy[a] * (T - L->T0) + L->accel[a];", "G[a] = L->buoy[a] * T + L->accel[a];",
     "Eq. 5: T - T0",
     "test_oracle_collision.py", "post_collision_momentum"),
    ("bounce_back_index", "lbm_oracle.c",
     "L->flow_bc[faces[a]] == BC_WALL) return fp[(long)io * S->ns + here];",
     "L->flow_bc[faces[a]] == BC_WALL) return fp[(long)i * S->ns + here];",
     "bounce-back reads the population itself, not its opposite",
     "test_oracle_cavity.py", "conserves_mass"),
    ("moving_wall_sign", "lbm_oracle.c",
     "return fp[(long)io * S->ns + here] + 2.0 * D->w[i] * L->rho0 * eu / CS2;",
     "return fp[(long)io * S->ns + here] - 2.0 * D->w[i] * L->rho0 * eu / CS2;",
     "moving-wall correction with the wrong sign",
     "test_oracle_closed_forms.py", "couette"),
    ("dirichlet_sign", "lbm_oracle.c",
     "return -gp[(long)io * S->ns + here] + 2.0 * om * c * L->face_T[face];",
     "return gp[(long)io * S->ns + here] + 2.0 * om * c * L->face_T[face];",
     "anti-bounce-back without its minus sign",
     "test_oracle_enthalpy.py", "two_region_melting"),
    ("neq_varpi_dropped", "lbm_oracle.c",
     "neq[4] = T * varpi * sigma;", "neq[4] = T * sigma;",
     "Eq. 37: varpi in n4_eq",
     "test_oracle_lattice.py", "geq_moments_and_neq"),
    ("neq_index", "lbm_oracle.c",
     "neq[1] = T * u[0];", "neq[1] = T * u[1];",
     "Eq. 37: n1_eq with the wrong velocity component",
     "test_oracle_lattice.py", "geq_moments_and_neq"),
    ("geq_weight", "lbm_oracle.c",
     "double om = i == 0 ? 1.0 - varpi : varpi / 6.0;",
     "double om = i == 0 ? 1.0 - varpi : varpi / 3.0;",
     "Eq. 42: omega_i of the moving directions",
     "test_oracle_lattice.py", "geq_moments_and_neq"),
    ("thermal_rate_swapped", "lbm_oracle.c",
     "zeta[1] = zeta[2] = zeta[3] = zeta_alpha;", "zeta[1] = zeta[2] = zeta[3] = L->zeta_T;",
     "Eq. 38: the diffusive rate on the heat-flux moments",
     "test_oracle_enthalpy.py", "two_region_melting"),
    ("thermal_sigma_dropped", "lbm_oracle.c",
     "return 1.0 / (0.5 + alpha_e / (L->sigma * csT2));",
     "return 1.0 / (0.5 + alpha_e / csT2);",
     "Eq. 41: sigma in zeta_alpha",
     "test_oracle_closed_forms.py", "temperature_wave"),
    ("m19_row_sign", "lbm_oracle.c",
     "{0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},",
     "{0, 4, -4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},",
     "Eq. A2: the q_x row with its signs flipped",
     "test_oracle_lattice.py", "moment_polynomials"),
    ("w19_swapped", "lbm_oracle.c",
     "1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,",
     "1.0 / 18, 1.0 / 36, 1.0 / 18, 1.0 / 36, 1.0 / 36,",
     "weights under Eq. 24: a face and an edge weight exchanged",
     "test_oracle_lattice.py", "weights_isotropy"),
    ("ninv7_entry", "lbm_oracle.c",
     "{0, 0.5, 0, 0, 1.0 / 6, 1.0 / 6, 1.0 / 6},", "{0, 0.5, 0, 0, 1.0 / 6, 1.0 / 6, -1.0 / 3},",
     "Eq. 43: one entry of N^-1",
     "test_oracle_lattice.py", "Ninv_as_printed"),
    ("periodic_wrap", "lbm_oracle.c",
     "fc >= 0 && L->flow_bc[fc] == BC_PERIODIC) {\n            c[a] = (c[a] + n[a]) % n[a];",
     "fc >= 0 && L->flow_bc[fc] == BC_PERIODIC) {\n            c[a] = (c[a] + n[a] - 1) % n[a];",
     "periodic wrap off by one site",
     "test_oracle_closed_forms.py", "shear_wave"),
    ("liquid_fraction_flipped", "lbm_oracle.c",
     "*fl = frac;", "*fl = 1.0 - frac;",
     "Eq. B9: the liquid fraction of the mushy range",
     "test_oracle_enthalpy.py", "enthalpy_state_relations"),
    ("viscosity_mapping", "__init__.py",
     "inv_s_nu = 0.5 + Ma * J * L * math.sqrt(3.0 * Pr) / math.sqrt(Ra)",
     "inv_s_nu = 0.5 + Ma * J * L * math.sqrt(Pr) / math.sqrt(Ra)",
     "Eq. 56: the 3 under the square root",
     "test_oracle_paper_tables.py", "halfway"),
    ("nusselt_first_order", "__init__.py",
     "q = (8.0 * T_wall - 9.0 * t0 + t1) / 3.0 * L / dT",
     "q = 2.0 * (T_wall - t0) * L / dT",
     "Eq. 53 on a halfway wall from a one-sided first-order gradient",
     "test_oracle_paper_channel.py", "formula"),
    ("geq_enthalpy_half", "lbm_oracle.c",
     "geq[i] = L->varpi * L->c_ref * T / 6.0 + 0.5 * eu * L->c_pl * T;",
     "geq[i] = L->varpi * L->c_ref * T / 6.0 + eu * L->c_pl * T;",
     "Eq. B12: the 1/2 of the advective part",
     "test_oracle_enthalpy.py", "geq_b12"),
    ("latent_heat_porosity_dropped", "lbm_oracle.c",
     "double El = L->sigma_l * L->c_pl * L->T_l + phi * L->L_a;",
     "double El = L->sigma_l * L->c_pl * L->T_l + L->L_a;",
     "Eq. B8: phi of the latent heat",
     "test_oracle_enthalpy.py", "latent"),
    ("matrix_diffusivity_swapped", "lbm_oracle.c",
     ": phi * L->alpha_f + (1.0 - phi) * L->alpha_m;",
     ": phi * L->alpha_m + (1.0 - phi) * L->alpha_f;",
     "alpha_e = phi alpha_f + (1 - phi) alpha_m with the two diffusivities exchanged",
     "test_oracle_closed_forms.py", "temperature_wave"),
    ("buoyancy_sign", "__init__.py",
     "buoy[gaxis] = -gsign * gbeta", "buoy[gaxis] = gsign * gbeta",
     "Eq. 5: buoyancy along gravity instead of against it",
     "test_oracle_cavity.py", "hot_fluid"),
    ("cavity_buoyancy_scale", "__init__.py",
     "gbeta = (Ma * math.sqrt(CS2)) ** 2 / (dT * L)", "gbeta = Ma ** 2 * CS2 / dT",
     "Eq. 56: u_c^2 = g beta dT L without the L",
     "test_oracle_paper_tables.py", "halfway"),
    ("darcy_number_scale", "__init__.py",
     "K = float(Da) * L * L if Da is not None else math.inf",
     "K = float(Da) * L if Da is not None else math.inf",
     "Da = K / L^2 read as K / L",
     "test_oracle_cavity.py", "x_mirror_symmetry"),
    ("channel_viscosity_mapping", "__init__.py",
     "inv_s_nu = 0.5 + J * L * u0 / (CS2 * Re)", "inv_s_nu = 0.5 + J * L * u0 / Re",
     "Eq. 51: c_s^2 dropped",
     "test_oracle_d3q15.py", "paper_channel_second_order"),
    ("stilde15_coefficient", "lbm_oracle.c",
     "S[1] = 2.0 * rho0 * uF / phi;", "S[1] = 1.0 * rho0 * uF / phi;",
     "Eq. 17: the energy-moment coefficient of D3Q15",
     "test_oracle_d3q15.py", "forcing_is_the_derivative"),
    ("meq15_coefficient", "lbm_oracle.c",
     "meq[4] = -7.0 / 3.0 * rho0 * ux;", "meq[4] = -2.0 / 3.0 * rho0 * ux;",
     "Eq. 15: the D3Q15 heat-flux moment with the D3Q19 coefficient",
     "test_oracle_d3q15.py", "equilibrium_moments"),
    ("node_wall_density", "lbm_oracle.c",
     "double rhob = out > 0.0 ? L->rho0 : m[0];", "double rhob = m[0];",
     "node walls: the withdrawing wall takes the fluid node's density",
     "test_oracle_nee.py", "steady_mass"),
    ("node_wall_flow_sign", "lbm_oracle.c",
     "for (int i = 0; i < D->q; ++i) f[i] += eb[i] - ef[i];",
     "for (int i = 0; i < D->q; ++i) f[i] += ef[i] - eb[i];",
     "node walls: the equilibrium parts exchanged with the wrong sign",
     "test_oracle_nee.py", "couette_between_node_walls"),
    ("node_wall_thermal_sign", "lbm_oracle.c",
     "for (int i = 0; i < Q7; ++i) g[i] += gb[i] - gf[i];",
     "for (int i = 0; i < Q7; ++i) g[i] += gf[i] - gb[i];",
     "node walls: the thermal equilibrium parts exchanged with the wrong sign",
     "test_oracle_nee.py", "conduction_between_node_walls"),
    ("kozeny_carman_exponent", "lbm_oracle.c",
     "double kc = p * p * p / ((1.0 - p) * (1.0 - p));",
     "double kc = p * p / ((1.0 - p) * (1.0 - p));",
     "Eq. 6: phi^2 in place of phi^3 in the Kozeny-Carman permeability",
     "test_oracle_closed_forms.py", "porosity_field"),
    ("ergun_field_exponent", "lbm_oracle.c",
     "*Fphi = L->F_phi < 0 ? 1.75 / sqrt(150.0 * p * p * p) : L->F_phi;",
     "*Fphi = L->F_phi < 0 ? 1.75 / sqrt(150.0 * p * p) : L->F_phi;",
     "Eq. 6: phi^2 in place of phi^3 in Ergun's coefficient of a field site",
     "test_oracle_closed_forms.py", "porosity_field"),
    ("outflow_anchor_dropped", "lbm_oracle.c",
     "if (via[i]) f[i] += D->w[i] * (L->rho0 - rho) / wsum;", "if (via[i]) f[i] += 0.0;",
     "reading 19: the outlet's pressure anchor left out",
     "test_oracle_closed_forms.py", "outflow_mass_balance"),
    ("enthalpy_diffusivity_swapped", "lbm_oracle.c",
     "(fl * L->alpha_l + (1.0 - fl) * L->alpha_s)", "(fl * L->alpha_s + (1.0 - fl) * L->alpha_l)",
     "Eq. B11: the liquid and solid diffusivities exchanged",
     "test_oracle_enthalpy.py", "two_region_melting"),
    ("velocity_sum_range", "lbm_oracle.c",
     "for (int i = 0; i < D->q; ++i) s += D->e[a * D->q + i] * f[i];",
     "for (int i = 0; i < 9; ++i) s += D->e[a * D->q + i] * f[i];",
     "Eq. 28 with its printed upper limit 8 taken literally",
     "test_oracle_lattice.py", "velocity_solves_eq26"),
    ("enthalpy_flow_gate", "lbm_oracle.c",
     "if (L->enthalpy && (L->flow_off || fl < 0.5)) {",
     "if (L->enthalpy && (L->flow_off || fl < 0.05)) {",
     "reading 22: the flow gate at f_l = 0.05 instead of 1/2",
     "test_oracle_enthalpy.py", "flow_gate"),
]


@pytest.fixture(scope="module")
def oracle_src():
    src = os.path.join(ROOT, "oracle")
    return {f: open(os.path.join(src, f)).read() for f in ("lbm_oracle.c", "__init__.py")}


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(mutant, oracle_src, tmp_path):
    name, fname, text, planted, _why, pin_file, pin_test = mutant
    assert oracle_src[fname].count(text) == 1, f"{name}: the planted line no longer matches"
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("_lib", "__pycache__"))
    (pkg / fname).write_text(oracle_src[fname].replace(text, planted))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pin_file), "-x", "-q",
                        "-m", "not gpu", "-k", pin_test, "-p", "no:cacheprovider"],
                       cwd=ROOT, env=dict(os.environ, LBM_ORACLE_UNDER_TEST=str(tmp_path)),
                       capture_output=True, text=True, timeout=600)
    # exit code 1: tests ran and one failed (2-5 would be an error, no tests, ...)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.returncode, r.stdout[-600:])
