"""The oracle's pins against plausible mistakes: each case plants one mistake
in a copy of lbm13_oracle.c (a flipped sign, a dropped term, a transposed
operand, a wrong index or rate), builds it on the CPU, and runs the oracle's
pin tests against that build; at least one pin must fail.

Two plausible alternatives are known to pass every pin and are not listed:
evaluating the equilibria at j instead of j + F/2 (reading R9: it moves only
the non-conserved moments by O(F), below every pin's tolerance), and a
quadratic instead of a linear extrapolation of the wall density (reading R12:
a change at second order in the node spacing).  The GPU path is held to the
oracle on both by the parity tests."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm13_oracle.c")
PINS = ["tests/test_oracle_basis.py", "tests/test_oracle_collision.py", "tests/test_oracle_linear.py",
        "tests/test_oracle_flows.py", "tests/test_oracle_waves.py"]

# name: (text in lbm13_oracle.c, planted replacement)
MUTANTS = {
    "q_sign_as_printed": ("case K_QX:  return x * (-3.0 + r2);", "case K_QX:  return x * (3.0 + r2);"),
    "h1_drops_E0_term": ("L->h1 = 17.0 / 26.0 - c1 / 2.0 - E0 / 13.0;", "L->h1 = 17.0 / 26.0 - c1 / 2.0;"),
    "h1_sign_in_q_eq": ("meq[K_QY] = jy * (p->c1 + L->h1 * rho + L->k1 * E);",
                        "meq[K_QY] = jy * (p->c1 - L->h1 * rho + L->k1 * E);"),
    "sigma_q_sign": ("L->sigma_q = -1309.0 / 2.0 * L->sigma_XX * L->A / L->B;",
                     "L->sigma_q = 1309.0 / 2.0 * L->sigma_XX * L->A / L->B;"),
    "c_erho_drops_term": ("L->c_erho = 140.0 + 28.0 * ceE + L->A * L->B / (22984.0 * p->Pr);",
                          "L->c_erho = 140.0 + L->A * L->B / (22984.0 * p->Pr);"),
    "inverse_not_transposed": ("Minv[j][k] = M[k][j] / d;", "Minv[j][k] = M[j][k] / d;"),
    "velocity_index_swapped": ("static const int vx_of[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1, 2, 0, -2, 0};",
                               "static const int vx_of[Q] = {0, 1, 0, -1, 0, 1, -1, 1, -1, 2, 0, -2, 0};"),
    "r_rate_from_XXe": ("L->s[K_RX] = L->s[K_RY] = p->s_r;", "L->s[K_RX] = L->s[K_RY] = p->s_XXe;"),
    "force_work_doubled": ("ms[K_E] = E + 13.0 * (", "ms[K_E] = E + 26.0 * ("),
    "energy_source_halved": ("/ rho + 26.0 * q;", "/ rho + 13.0 * q;"),
    "anti_bounce_back_sign": ("out = -val + 2.0 * feq_part(L, &ws, j, 0);", "out = val + 2.0 * feq_part(L, &ws, j, 0);"),
    "bounce_back_correction_sign": ("out = val - 2.0 * feq_part(L, &ws, j, 1);    /* bounce-back",
                                    "out = val + 2.0 * feq_part(L, &ws, j, 1);    /* bounce-back"),
    "two_link_lands_on_same_row": ("lx = (int)lround(x + (2.0 * a - 1.0) * vx_of[j]);\n"
                                   "                    ly = (int)lround(y + (2.0 * a - 1.0) * vy_of[j]);\n"
                                   "                    normal_link = vy_of[j] == 0;",
                                   "lx = x;\n"
                                   "                    ly = (int)lround(y + (2.0 * a - 1.0) * vy_of[j]);\n"
                                   "                    normal_link = vy_of[j] == 0;"),
    "wall_density_not_extrapolated": ("s.rho = 1.5 * r0 - 0.5 * r1;", "s.rho = r0;"),
    "wall_energy_drops_kinetic_part": ("s.E = s.rho * (26.0 * w->T - 28.0) + 13.0 * s.rho * (s.ux * s.ux + s.uy * s.uy);",
                                       "s.E = s.rho * (26.0 * w->T - 28.0);"),
    "nusselt_kappa_inverted": ("double kappa = L->p.nu / L->p.Pr;", "double kappa = L->p.nu * L->p.Pr;"),
    "corner_at_mean_wall_data": ("val - 2.0 * feq_part(L, &a, j, 1) - 2.0 * feq_part(L, &b, j, 1);",
                                 "val - 2.0 * feq_part(L, &(wall_state){0.5 * (a.rho + b.rho), "
                                 "0.5 * (a.E + b.E), 0.5 * (a.ux + b.ux), 0.5 * (a.uy + b.uy)}, j, 1);"),
    "corner_one_wall_only": ("val - 2.0 * feq_part(L, &a, j, 1) - 2.0 * feq_part(L, &b, j, 1);",
                             "val - 2.0 * feq_part(L, &b, j, 1);"),
    "north_wall_second_node_misplaced": ("else                { y0 = L->ny - 1;  y1 = L->ny - 2;  x0 = x1 = pos; }",
                                         "else                { y0 = L->ny - 1;  y1 = L->ny - 3;  x0 = x1 = pos; }"),
    "east_corners_take_west_wall_data": ("int sx = tx < 0 ? 0 : 1, sy = ty < 0 ? 2 : 3;",
                                         "int sx = 0, sy = ty < 0 ? 2 : 3;"),
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of {name} not found once"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    lib = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(lib), str(c), "-lm"])
    env = dict(os.environ, LBM13_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, f"{name}: no pin failed\n{r.stdout[-1500:]}"
    assert "failed" in r.stdout.splitlines()[-1]
