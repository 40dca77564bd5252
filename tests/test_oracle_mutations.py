"""Mutation checks of the oracle's pins (CPU only).

Each case plants one plausible mistake in a copy of oracle/lbref.c:
- a flipped sign;
- a swapped operand or component;
- a dropped factor or term;
- a wrong neighbour.

The copy is compiled apart. The pin meant to catch the mistake then runs in
a subprocess against that build (the oracle's loader takes the library named
by LBREF_LIB), and it must fail there. On the real oracle it passes, in the
rest of the suite. The real oracle source is read, never changed."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbref.c")

FLUID = "tests/test_oracle_fluid.py::"
PART = "tests/test_oracle_particles.py::"
LATT = "tests/test_oracle_lattice.py::"

# name: ([(old, new, occurrences)], pins that must fail)
MUTANTS = {
    "colour rule components swapped": (
        [("if (dr > 0)\n            rn[0] += dr;\n        else\n            rn[1] += fabs(dr);",
          "if (dr > 0)\n            rn[1] += dr;\n        else\n            rn[0] += fabs(dr);", 1)],
        [PART + "test_colour_rule_sign"]),
    "walls keep psi = 0": (
        [("if (cnt == 0) {\n            c->psi[n] = 0.0;",
          "if (cnt == 0 || c->type[n] == T_WALL) {\n            c->psi[n] = 0.0;", 1)],
        [FLUID + "test_walls_leave_a_uniform_mixture_at_rest"]),
    "Shan-Chen force sign": (
        [("-g * pc * s", "g * pc * s", 3)],
        [FLUID + "test_demixing_sign_of_coupling"]),
    "weighted Shan-Chen stencil": (
        [("double ps = c->psi[co * N + m];", "double ps = WV[i] * c->psi[co * N + m];", 1)],
        [FLUID + "test_bruteforce_one_step_fluid"]),
    "shifted velocity without the 1/tau weights": (
        [("num[k] += c->jm[(cc * 3 + k) * N + n] / t;", "num[k] += c->jm[(cc * 3 + k) * N + n];", 1),
         ("den += c->rho[cc * N + n] / t;", "den += c->rho[cc * N + n];", 1)],
        [FLUID + "test_bruteforce_one_step_fluid"]),
    "force enters the equilibrium velocity with the wrong sign": (
        [("up[k] + t * c->frc", "up[k] - t * c->frc", 1)],
        [FLUID + "test_body_force_momentum_rate"]),
    "equilibrium second-order coefficient": (
        [("4.5 * cu * cu", "4.0 * cu * cu", 1)],
        [LATT + "test_equilibrium_moments"]),
    "pull streaming from the wrong neighbour": (
        [("long src = i == 0 ? y : neighbour(c, x0, y0, z0, OPPV[i]);",
          "long src = i == 0 ? y : neighbour(c, x0, y0, z0, i);", 1)],
        [FLUID + "test_bruteforce_one_step_fluid"]),
    "moving bounce-back term C with the wrong sign": (
        [("double C = 6.0 * WV[i] * c->rho[cc * N + y] * uc;",
          "double C = -6.0 * WV[i] * c->rho[cc * N + y] * uc;", 1)],
        [PART + "test_co_moving_fluid_is_left_at_equilibrium_exactly"]),
    "momentum exchange without the factor 2": (
        [("F[k] = (2.0 * fr + C) * CV[io][k];", "F[k] = (fr + C) * CV[io][k];", 1)],
        [PART + "test_momentum_conservation_free_particle"]),
    "link torque operands swapped": (
        [("cross(rb, F, T);", "cross(F, rb, T);", 1)],
        [PART + "test_rotating_sphere_torque_opposes_spin"]),
    "covered node's momentum with the wrong sign": (
        [("P->Fpend[k] += mom[k];", "P->Fpend[k] -= mom[k];", 1)],
        [PART + "test_momentum_conservation_free_particle"]),
    "lubrication pulls the particles together": (
        [("A->Fpair[k] -= s * rh[k];\n                    B->Fpair[k] += s * rh[k];",
          "A->Fpair[k] += s * rh[k];\n                    B->Fpair[k] -= s * rh[k];", 1)],
        [PART + "test_lubrication_sphere_limit"]),
    "lubrication without the reduced-mass cap": (
        [("if (gam > mred) gam = mred;", "", 1)],
        [PART + "test_lubrication_capped_at_reduced_mass[1.0]"]),
    "Hertz strength with the wrong power of sigma": (
        [("double ebar = k_hertz * pow(sbar, 2.5);", "double ebar = k_hertz * pow(sbar, 1.5);", 1)],
        [PART + "test_sphere_limit_is_hertz"]),
    "explicit Euler instead of the velocity-first update": (
        [("vel[k] += force[k] / mass;\n        pos[k] += vel[k];",
          "pos[k] += vel[k];\n        vel[k] += force[k] / mass;", 1)],
        [PART + "test_translation_closed_form"]),
    "rotation composed on the wrong side": (
        [("qmul(quat, dq, qn);", "qmul(dq, quat, qn);", 1)],
        [PART + "test_symmetric_top_free_precession"]),
    "surface velocity without the rotation": (
        [("cross(P->W, rb, wr);\n                for (int k = 0; k < 3; k++) us[k] = P->V[k] + wr[k];",
          "cross(P->W, rb, wr);\n                for (int k = 0; k < 3; k++) us[k] = P->V[k];", 1)],
        [FLUID + "test_bruteforce_one_step_static_particle"]),
    "torque arm from the wrong centre": (
        [("double rb[3] = {node_disp(c, 0, x0, P->X[0]) - 0.5 * CV[i][0],",
          "double rb[3] = {node_disp(c, 0, x0, P->X[0] + 1.0) - 0.5 * CV[i][0],", 1)],
        [FLUID + "test_bruteforce_one_step_static_particle"]),
    "wall bounce-back into the incoming slot": (
        [("fn[((long)cc * Q + i) * N + y] = c->fs[((long)cc * Q + io) * N + y];",
          "fn[((long)cc * Q + i) * N + y] = c->fs[((long)cc * Q + i) * N + y];", 1)],
        [FLUID + "test_bruteforce_one_step_fluid"]),
    "shell fill divides by 18, not by the fluid neighbours": (
        [("double rn[2] = {s[0] / cnt, s[1] / cnt};", "double rn[2] = {s[0] / 18.0, s[1] / 18.0};", 1)],
        [FLUID + "test_walls_leave_a_uniform_mixture_at_rest"]),
    "C with the other component's density": (
        [("double C = 6.0 * WV[i] * c->rho[cc * N + y] * uc;",
          "double C = 6.0 * WV[i] * c->rho[(1 - cc) * N + y] * uc;", 1)],
        [FLUID + "test_bruteforce_one_step_static_particle"]),
    "Shan-Chen sum over the own component": (
        [("double ps = c->psi[co * N + m];", "double ps = c->psi[cc * N + m];", 1)],
        [FLUID + "test_bruteforce_one_step_fluid"]),
    "Hertz force applied with the same sign to both particles": (
        [("B->Fpair[k] += fj[k];\n                A->Fpair[k] -= fj[k];",
          "B->Fpair[k] += fj[k];\n                A->Fpair[k] += fj[k];", 1)],
        [PART + "test_hertz_pair_force_applied_to_both_particles"]),
    "Hertz torques of the two particles exchanged": (
        [("A->Tpair[k] += ti[k];\n                B->Tpair[k] += tj[k];",
          "A->Tpair[k] += tj[k];\n                B->Tpair[k] += ti[k];", 1)],
        [PART + "test_hertz_pair_force_applied_to_both_particles"]),
    "inside test in the lab frame's transpose": (
        [("d[k] = R[0][k] * dx[0] + R[1][k] * dx[1] + R[2][k] * dx[2];",
          "d[k] = R[k][0] * dx[0] + R[k][1] * dx[1] + R[k][2] * dx[2];", 1)],
        [PART + "test_coverage_matches_exact_rational_count", FLUID + "test_bruteforce_one_step_static_particle"]),
    "inside test with the radii exchanged": (
        [("double ip2 = 1.0 / (rp * rp), io2 = 1.0 / (ro * ro);",
          "double ip2 = 1.0 / (ro * ro), io2 = 1.0 / (rp * rp);", 1)],
        [PART + "test_coverage_matches_exact_rational_count"]),
    "uncovered node at the particle's translation only": (
        [("cross(P->W, r, wr);\n            for (int k = 0; k < 3; k++) us[k] = P->V[k] + wr[k];",
          "cross(P->W, r, wr);\n            for (int k = 0; k < 3; k++) us[k] = P->V[k];", 1)],
        [PART + "test_uncovered_node_gets_the_local_equilibrium"]),
    "uncovered node's density over neighbours the particle now covers": (
        [("if (m < 0 || c->type[m] != T_FLUID || c->nowner[m] >= 0) continue;",
          "if (m < 0 || c->type[m] != T_FLUID) continue;", 1)],
        [PART + "test_uncovered_node_gets_the_local_equilibrium"]),
    "prescribed rotation about the body-frame axis": (
        [("for (int k = 0; k < 3; k++) wb[k] = R[0][k] * W[0] + R[1][k] * W[1] + R[2][k] * W[2];",
          "for (int k = 0; k < 3; k++) wb[k] = W[k];", 1)],
        [PART + "test_prescribed_motion_closed_form"]),
    "gyroscopic term with the wrong sign": (
        [("cross(wb, L, wl);", "cross(L, wb, wl);", 1)],
        [PART + "test_symmetric_top_free_precession"]),
}


@pytest.fixture(scope="module")
def gcc():
    exe = shutil.which("gcc")
    if not exe:
        pytest.skip("gcc not found")
    return exe


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_planted_mistake(name, gcc, tmp_path):
    edits, pins = MUTANTS[name]
    src = open(SRC).read()
    for old, new, count in edits:
        assert src.count(old) == count, f"{name}: the planted edit no longer matches the oracle"
        src = src.replace(old, new)
    (tmp_path / "lbref.c").write_text(src)
    shutil.copy(os.path.join(ROOT, "oracle", "lbref.h"), tmp_path / "lbref.h")
    lib = tmp_path / "liblbref_mutant.so"
    subprocess.check_call([gcc, "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           str(tmp_path / "lbref.c"), "-o", str(lib), "-lm"])
    env = dict(os.environ, LBREF_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    # exit status 1: tests ran and at least one failed (not a collection error)
    assert r.returncode == 1, f"{name} was not caught:\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}"
