"""Plants plausible mistakes in copies of the oracle source (on the CPU) and checks
that the pins of test_oracle_pins.py catch every one of them."""
import os

import pytest

import oracle
import test_oracle_pins as P
from conftest import golden_rows
from paper_2502_16818_gb300 import workloads as W


def _g():
    return golden_rows


PINS = {
    "feq_moments": lambda: [P.test_feq_reproduces_maxwellian_moments("sod", W.VSET_SOD, 0.0),
                            P.test_feq_reproduces_maxwellian_moments("tgv", W.VSET_TGV, 3.0)],
    "central_moments": lambda: [P.test_central_moments_match_quadrature(3.0, 1.7),
                                P.test_central_moments_match_quadrature(0.0, 0.8)],
    "macros_single": lambda: [P.test_macros_of_single_velocity("tgv", W.VSET_TGV)],
    "minmod_golden": lambda: [P.test_minmod_eq16(_g())],
    "nnd_golden": lambda: [P.test_nnd_hand_evaluations(_g())],
    "relaxation": lambda: [P.test_pure_relaxation_factor(0)],
    "conservation": lambda: [P.test_global_conservation_periodic(0)],
    "anisotropic": lambda: [P.test_sound_speed_anisotropic_cells("x"),
                            P.test_sound_speed_anisotropic_cells("y")],
    "solve40": lambda: [P.test_solve_against_40_digit_solution("tgv", W.VSET_TGV)],
    "tne_zero": lambda: [P.test_tne_zero_at_equilibrium_and_trace_identity()],
    "tne_brute": lambda: [P.test_tne_brute_force_cell()],
    "velocity_set": lambda: [P.test_velocity_set_eq2(_g())],
    "matrix_columns": lambda: [P.test_central_matrix_columns_are_monomials_of_peculiar_velocity()],
    "sound": lambda: [P.test_sound_speed_1d(3.0)],
}

# (label, original text, planted text, pins expected to catch it)
MUTANTS = [
    ("rows 11 and 12 swapped", "M[10 * NV + i] = cx * cx * cy;\n        M[11 * NV + i] = cx * cy * cy;",
     "M[10 * NV + i] = cx * cy * cy;\n        M[11 * NV + i] = cx * cx * cy;", ["matrix_columns", "tne_brute"]),
    ("peculiar velocity with +u", "double cx = vx[i] - ux;", "double cx = vx[i] + ux;", ["feq_moments"]),
    ("equilibrium in the lab frame", "orc_central_matrix(vx, vy, eta, ux, uy, M);\n    orc_central_moments_eq",
     "orc_central_matrix(vx, vy, eta, 0.0, 0.0, M);\n    orc_central_moments_eq", ["feq_moments"]),
    ("fourth moment (K+1) T^2", "fbar[13] = rho * (K + 2.0) * T * T;", "fbar[13] = rho * (K + 1.0) * T * T;",
     ["central_moments"]),
    ("K without I", "const double K = 2.0 + I;\n    for (int k = 0; k < NV; ++k) fbar[k] = 0.0;",
     "const double K = 2.0;\n    for (int k = 0; k < NV; ++k) fbar[k] = 0.0;", ["central_moments"]),
    ("temperature without eta", "e += f[i] * (cx * cx + cy * cy + eta[i] * eta[i]);",
     "e += f[i] * (cx * cx + cy * cy);", ["macros_single", "sound"]),
    ("minmod keeps the larger", "return (fabs(X) <= fabs(Y)) ? X : Y;", "return (fabs(X) <= fabs(Y)) ? Y : X;",
     ["minmod_golden"]),
    ("minmod ignores signs", "if ((X > 0.0) != (Y > 0.0)) return 0.0;", "", ["minmod_golden"]),
    ("NND drops the 1/2", "double HLp = fp[2] + 0.5 * orc_minmod(dp[2], dp[1]);",
     "double HLp = fp[2] + orc_minmod(dp[2], dp[1]);", ["nnd_golden"]),
    ("NND sign", "return ((HLp + HRp) - (HLm + HRm)) / dr;", "return ((HLm + HRm) - (HLp + HRp)) / dr;",
     ["nnd_golden"]),
    ("f+ and f- swapped", "fp[k] = 0.5 * (v + fabs(v)) * fs[k];\n        fm[k] = 0.5 * (v - fabs(v)) * fs[k];",
     "fp[k] = 0.5 * (v - fabs(v)) * fs[k];\n        fm[k] = 0.5 * (v + fabs(v)) * fs[k];", ["nnd_golden"]),
    ("H_R uses the wrong interface", "double HRp = fm[3] - 0.5 * orc_minmod(dm[2], dm[3]);",
     "double HRp = fm[3] - 0.5 * orc_minmod(dm[1], dm[2]);", ["nnd_golden"]),
    ("RK stage 2 restarts from f", "f[k] = 0.5 * f[k] + 0.5 * (g[k] + p->dt * L[k]);",
     "f[k] = 0.5 * f[k] + 0.5 * (f[k] + p->dt * L[k]);", ["relaxation"]),
    ("collision sign", "L[i * plane + c] = -adv - (fc[i] - feq[i]) / p->tau;",
     "L[i * plane + c] = -adv + (fc[i] - feq[i]) / p->tau;", ["relaxation"]),
    ("periodic ghost reflects", "        j %= n;\n        return j < 0 ? j + n : j;",
     "        j %= n;\n        return j < 0 ? -j : j;", ["conservation"]),
    ("y derivative with dx", "orc_nnd_derivative(vy[i], sy, p->dy)", "orc_nnd_derivative(vy[i], sy, p->dx)",
     ["anisotropic"]),
    ("forward substitution ignores the row permutation", "double acc = rhs[perm[i]];",
     "double acc = rhs[i];", ["solve40", "feq_moments"]),
    ("TNE of f instead of f - f_eq", "acc += (fc[i] - feq[i]) * M[k * NV + i];",
     "acc += fc[i] * M[k * NV + i];", ["tne_zero", "tne_brute"]),
    ("TNE rows shifted", "out[(k - 4) * plane + c] = acc;", "out[(k == 15 ? 4 : k - 3) * plane + c] = acc;",
     ["tne_brute"]),
    ("diagonal member order", "static const double diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};",
     "static const double diag[4][2] = {{1, 1}, {-1, -1}, {-1, 1}, {1, -1}};", ["velocity_set"]),
]


@pytest.mark.parametrize("label,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, label, old, new, pins):
    src = oracle.source()
    assert src.count(old) == 1, "mutation anchor not unique: %s" % label
    path = oracle.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), "mutant.so"))
    caught = []
    with oracle.use_library(path):
        for name in pins:
            try:
                PINS[name]()
            except (AssertionError, RuntimeError, ArithmeticError, ValueError, IndexError) as e:
                caught.append((name, type(e).__name__))
    assert caught, "no pin caught the planted mistake '%s'" % label
