"""Planted mistakes: each pin below must fail on a copy of the oracle with one plausible mistake
in its arithmetic (a dropped term, a wrong sign, index or coefficient, a transposed operand),
so that the pins are shown to see what they are meant to see. Every copy is compiled with the
oracle's own flags into tests/.mutants/ and the pin runs in a child process that loads it; the
same pins pass on the oracle itself in the rest of the suite. CPU only."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", ".mutants")
PINS = "tests/test_oracle_pins.py::"

# (name, text in the oracle, planted replacement, the pin that must fail)
MUTANTS = [
    ("newton_tolerance_loose", "#define NEWTON_TOL 1e-12", "#define NEWTON_TOL 1e-6",
     PINS + "test_riemann_star_pressure_to_the_newton_tolerance"),
    ("hugoniot_tolerance_loose", "#define HUGONIOT_TOL 1e-14", "#define HUGONIOT_TOL 1e-7",
     PINS + "test_mg_shock_density_to_the_hugoniot_tolerance"),
    ("rk2_level_set_average_dropped",
     "for (long c = 0; c < N; ++c) phi[c] = 0.5 * (phi[c] + (wk->phi1[c] + dt * wk->L[c]));",
     "for (long c = 0; c < N; ++c) phi[c] = (wk->phi1[c] + dt * wk->L[c]);",
     PINS + "test_smooth_entropy_wave_converges_at_second_order"),
    ("face_slope_not_halved", "tm[v] = Q[v] - 0.5 * s;\n    tp[v] = Q[v] + 0.5 * s;",
     "tm[v] = Q[v] - s;\n    tp[v] = Q[v] + s;", PINS + "test_smooth_entropy_wave_converges_at_second_order"),
    ("muscl_stencil_across_the_interface", "if (id[cm] != m || id[cp] != m) return;",
     "if (id[cm] != m && id[cp] != m) return;", PINS + "test_muscl_stencil_stops_at_the_interface"),
    ("hllc_star_energy_sign", "(Ss + pK / (rK * (SK - uK)))", "(Ss - pK / (rK * (SK - uK)))",
     PINS + "test_hllc_star_state_energy_satisfies_the_jump_condition"),
    ("fiver_other_side_star_density", "  S[0] = rs[3];", "  S[0] = rs[2];",
     PINS + "test_shock_bubble_is_mirror_symmetric"),
    ("level_set_upwind_reversed", "if (vel >= 0.0) return (2.0 * pp1", "if (vel < 0.0) return (2.0 * pp1",
     PINS + "test_level_set_residual_of_a_quartic_in_every_axis"),
    ("level_set_w_term_sign", "Lphi[c] = -((u * Dx + v * Dy) + w * Dz);", "Lphi[c] = -((u * Dx + v * Dy) - w * Dz);",
     PINS + "test_level_set_residual_of_a_quartic_in_every_axis"),
    ("reinit_first_layer_not_held", "          if (first) {\n            nxt[c] = cur[c];\n            continue;\n          }\n",
     "", PINS + "test_reinit_holds_the_first_layer_and_moves_the_rest"),
    ("reinit_godunov_sum", "G2[d] = fmax(x * x, y * y);", "G2[d] = x * x + y * y;",
     PINS + "test_reinit_keeps_a_distance_with_ridges"),
    ("reinit_sign_of_the_iterate", "double S = phi0[c] / sqrt(phi0[c] * phi0[c] + h * h);",
     "double S = cur[c] / sqrt(cur[c] * cur[c] + h * h);", PINS + "test_two_reinit_iterations_in_closed_form"),
    ("phase_update_face_rule_dropped",
     "        for (int d = 0; d < 3; ++d)\n          for (int sgn = -1; sgn <= 1; sgn += 2) {",
     "        for (int d = 0; d < 0; ++d)\n          for (int sgn = -1; sgn <= 1; sgn += 2) {",
     PINS + "test_phase_update_takes_face_neighbours_before_the_26_neighbourhood"),
    ("mg_fixed_node_shifted", "int st = mg_rk4_substep(q, K->p - i * K->dnode, -K->dnode, &rho, &fv);",
     "int st = mg_rk4_substep(q, K->p - (i + 1) * K->dnode, -K->dnode, &rho, &fv);",
     PINS + "test_mg_riemann_rarefactions_match_ode_integration"),
    ("mg_cutoff_pressure", "return q->prm[0] * q->prm[1] * q->prm[1] * q->prm[5];",
     "return q->prm[0] * q->prm[1] * q->prm[5];", PINS + "test_mg_riemann_rarefactions_match_ode_integration"),
    ("mg_dedrho_sign", "*de_drho = (deR - dpR / rg) * q->prm[0] / (rho * rho);",
     "*de_drho = (deR + dpR / rg) * q->prm[0] / (rho * rho);",
     PINS + "test_mg_shock_curve_slope_is_the_derivative_of_the_curve"),
    ("bisection_sides_swapped", "      if (F < 0.0) a = m; else b = m;", "      if (F > 0.0) a = m; else b = m;",
     PINS + "test_riemann_star_pressure_to_the_newton_tolerance"),
    ("sampler_fan_pressure", "        out[2] = pb * pow(cf / c, 2.0 * g / (g - 1.0)) - pc;\n      }\n    }\n  } else {",
     "        out[2] = pb * pow(cf / c, 2.0 * g / (g - 1.0)) + pc;\n      }\n    }\n  } else {",
     PINS + "test_exact_sampler_waves_satisfy_their_relations"),
    ("shock_speed_sign", "out[2] = (rs * out[1] - K.rho * K.u) / (rs - K.rho);",
     "out[2] = (rs * out[1] + K.rho * K.u) / (rs - K.rho);",
     PINS + "test_shock_speed_is_galilean_and_carries_the_momentum_jump"),
    ("rk3_stage_coefficient",
     "wk->W1[x] = (0.75 * W[x] + 0.25 * wk->W1[x]) + 0.25 * dt * wk->R[x];",
     "wk->W1[x] = (0.75 * W[x] + 0.25 * wk->W1[x]) + 0.5 * dt * wk->R[x];",
     "tests/test_oracle_scheme_variants.py::test_time_integrators_reach_their_order"),
    ("euler_level_set_coefficient", "for (long c = 0; c < N; ++c) phi[c] = phi[c] + dt * wk->L[c];",
     "for (long c = 0; c < N; ++c) phi[c] = phi[c] + 0.5 * dt * wk->L[c];",
     "tests/test_oracle_scheme_variants.py::test_forward_euler_converges_to_the_exact_translation"),
    ("mirror_about_the_cell_centre", "(bchi == BC_SYMMETRY ? 2 * n - 1 - i : n - 1)",
     "(bchi == BC_SYMMETRY ? 2 * n - 2 - i : n - 1)",
     "tests/test_oracle_symmetry.py::test_mirror_side_equals_the_symmetric_full_domain"),
    ("radial_source_off_centre", "double r = g->x0 + (i + 0.5) * g->h;", "double r = g->x0 + (i + 1.0) * g->h;",
     "tests/test_oracle_symmetry.py::test_steady_radial_flow_residual_vanishes_at_second_order"),
    ("nasg_lower_bound", "if (q->type == EOS_SG || q->type == EOS_NASG) return -q->prm[1];",
     "if (q->type == EOS_SG) return -q->prm[1];\n  if (q->type == EOS_NASG) return 0.0;",
     "tests/test_oracle_nasg.py::test_nasg_without_covolume_is_the_stiffened_gas_in_tension"),
    ("jwl_first_exponential_sign", "double x = R * rho0 / rho, ex = exp(-x)",
     "double x = R * rho0 / rho, ex = i == 0 ? exp(x) : exp(-x)",
     "tests/test_oracle_jwl.py::test_jwl_is_an_ideal_gas_at_low_density"),
    ("radial_source_energy_without_p", "acc[4] = acc[4] - a * (W[4 * N + c] + P[4 * N + c]);",
     "acc[4] = acc[4] - a * (W[4 * N + c]);",
     "tests/test_oracle_symmetry.py::test_steady_radial_flow_residual_vanishes_at_second_order"),
    ("phase_update_mirror_image_velocity", "                  prim_at(g, P, i + di, j + dj, k + dk, q);",
     "                  { long nb2 = cell_index(g, i + di, j + dj, k + dk);\n"
     "                    for (int v = 0; v < 5; ++v) q[v] = P[v * N + nb2]; }",
     "tests/test_oracle_symmetry.py::test_phase_update_across_a_mirror_side"),
    ("band_cutoff_coefficient", "(2.0 * a + gamma - 3.0 * beta)", "(2.0 * a + gamma - 2.0 * beta)",
     "tests/test_oracle_narrow_band.py::test_cutoff_closed_form"),
    ("band_clip_skipped", "  band_clip(g, phi); /* narrow band (Reading R38) */", "",
     "tests/test_oracle_narrow_band.py::test_values_beyond_the_outer_tube_are_clipped_and_held"),
]


def _build(name, old, new):
    src = open(O.SRC).read()
    assert src.count(old) == 1, name
    d = os.path.join(WORK, name)
    os.makedirs(d, exist_ok=True)
    path = os.path.join(d, "m2c_oracle.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(d, "libm2c_oracle.so")
    subprocess.run(["gcc", *O.CFLAGS, "-o", lib, path, "-lm"], check=True)
    return lib


def _run_pin(lib, pin):
    env = dict(os.environ, M2C_ORACLE_MUTANT_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", pin, "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr).strip().splitlines()[-1:]


def test_every_planted_mistake_fails_its_pin():
    os.makedirs(WORK, exist_ok=True)

    def one(m):
        name, old, new, pin = m
        lib = _build(name, old, new)
        code, tail = _run_pin(lib, pin)
        return name, pin, code, tail
    with ThreadPoolExecutor(4) as ex:
        results = list(ex.map(one, MUTANTS))
    # pytest exits 1 when a test failed; 0 would mean the pin missed the mistake, anything else
    # a collection or usage error
    missed = [(n, p, c, t) for n, p, c, t in results if c != 1]
    assert not missed, missed


@pytest.mark.parametrize("name,old,new,pin", MUTANTS[:1])
def test_the_pins_pass_on_the_oracle_itself(name, old, new, pin):
    """The control: the same child-process run on the unmodified oracle passes."""
    code, tail = _run_pin(O.build(), pin)
    assert code == 0, tail
