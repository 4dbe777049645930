"""Strength of the oracle's pins: plausible mistakes are planted, one at a
time, in a copy of the oracle's source (never in the oracle itself), the
copy is compiled on the CPU, and the CPU pins are run against it; every
planted mistake must make at least one pin fail.

The mistakes: a wrong kernel normalisation or derivative sign, a flipped
pressure force, the neighbour's stress dropped from Eq. 26, the colour
weight phi_i replaced by phi_j (Eq. 22), an arithmetic instead of a
harmonic pair viscosity (Eq. 13), the pressure difference of U* (Eq. 9)
reversed, the density update reversed (Eq. 6), the factor 2 of Eq. 6 dropped
(only the acoustic standing wave catches that one), the wall's mirror
pressure dropped, the wall volume doubled, v* = v_i instead of the wall's
velocity in the continuity equation, the wall's normal velocity not
mirrored in the Riemann state, the cross-phase penalty weight
4 phi_i phi_j halved (Eq. 33), the same-phase penalty of Eq. 33 halved or
dropped, its projection T-bar replaced by N-bar, the contraction of
Eq. 30 transposed (A^T A for A A^T), and the surface stress of Eq. 24 made
20% weak.  An unmodified copy passes the same
harness."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sph_oracle.c")
# the quick, targeted pins first: each copy stops at its first failing pin
PINS = ["test_oracle_kernel.py", "test_oracle_penalty_pair.py", "test_oracle_surface_force.py", "test_oracle_wall_pair.py",
        "test_oracle_riemann.py", "test_oracle_weights.py", "test_golden.py", "test_oracle_neighbors.py",
        "test_oracle_reading_flags.py", "test_oracle_periodic.py", "test_oracle_invariants.py",
        "test_oracle_acoustics.py", "test_oracle_dynamics.py"]

MUTANTS = {
    "kernel normalisation": ("return dim == 2 ? 7.0 / (4.0 * ORA_PI * h * h)",
                             "return dim == 2 ? 8.0 / (4.0 * ORA_PI * h * h)"),
    "kernel derivative sign": ("return -5.0 * wendland_alpha(dim, h) * q * t * t * t / h;",
                               "return 5.0 * wendland_alpha(dim, h) * q * t * t * t / h;"),
    "pressure force sign": ("a_p[d] += -2.0 / rho_i * Ps * gradW[d] * Vj;",
                            "a_p[d] += 2.0 / rho_i * Ps * gradW[d] * Vj;"),
    "neighbour stress dropped": ("? si->Pi[3 * a + b] + sj->Pi[3 * a + b] + (P->penalty_scope",
                                 "? si->Pi[3 * a + b] + si->Pi[3 * a + b] + (P->penalty_scope"),
    "same-phase penalty halved": ("(P->penalty_scope == 1 ? 0.0 : pen)", "(P->penalty_scope == 1 ? 0.0 : 0.5 * pen)"),
    "same-phase penalty dropped": ("(P->penalty_scope == 1 ? 0.0 : pen)", "(P->penalty_scope == 1 ? 0.0 : 0.0 * pen)"),
    "same-phase projection N-bar instead of T-bar": (
        "M[3 * a + b] = same ? 0.5 * (si->T[3 * a + b] + sj->T[3 * a + b])",
        "M[3 * a + b] = same ? 0.5 * (si->N[3 * a + b] + sj->N[3 * a + b])"),
    "penalty contraction transposed": ("s += P->penalty_form == 0 ? A[3 * a + c] * A[3 * b + c]",
                                       "s += P->penalty_form == 0 ? A[3 * c + a] * A[3 * c + b]"),
    "colour weight of j": ("g[d] += 2.0 * phi_i * Cij * pp->dW[k] * pp->e[3 * k + d] * Vj;",
                           "g[d] += 2.0 * (1.0 - phi_i) * Cij * pp->dW[k] * pp->e[3 * k + d] * Vj;"),
    "arithmetic pair viscosity": ("? 2.0 * P->eta[ki] * P->eta[kj] / (P->eta[ki] + P->eta[kj])",
                                  "? 0.5 * (P->eta[ki] + P->eta[kj])"),
    "U* pressure difference reversed": ("return (zl * L.U + zr * R.U + L.p - R.p) / (zl + zr);",
                                        "return (zl * L.U + zr * R.U - L.p + R.p) / (zl + zr);"),
    "density update reversed": ("rho[i] += dt * drho[i];", "rho[i] -= dt * drho[i];"),
    "continuity factor 2 dropped": ("            s *= 2.0 * rho_i;", "            s *= rho_i;"),
    "wall mirror pressure dropped": ("R.p = p_i; R.c = c0;\n                    pbar = pair_pbar(rho_i, p_i, rho_i, p_i);",
                                     "R.p = 0.0; R.c = c0;\n                    pbar = pair_pbar(rho_i, p_i, rho_i, 0.0);"),
    "cross-phase penalty weight halved": ("- 4.0 * phi_i * phi_j * pen;", "- 2.0 * phi_i * phi_j * pen;"),
    "own-fluid correction from i alone": (
        "t += 0.5 * (Bk[9 * i + 3 * a + b] + Bk[9 * j + 3 * a + b]) * gradW[b];",
        "t += Bk[9 * i + 3 * a + b] * gradW[b];"),
    "own-fluid correction over every neighbour": (
        "if (own_fluid && S->kind[j] != S->kind[i]) continue;", "(void)own_fluid;"),
    "cross-phase stress weights swapped": (
        ": 2.0 * phi_j * si->Pi[3 * a + b] + 2.0 * phi_i * sj->Pi[3 * a + b])",
        ": 2.0 * phi_i * si->Pi[3 * a + b] + 2.0 * phi_j * sj->Pi[3 * a + b])"),
    "wall v* = v_i in continuity": ("                    for (int d = 0; d < dim; ++d) vs[d] = vj[d];",
                                    "                    for (int d = 0; d < dim; ++d) vs[d] = vi[d];"),
    "wall velocity not mirrored": ("R.U = 2.0 * Uw - L.U;", "R.U = Uw;"),
    "surface stress 20% weak": ("st->Pi[3 * a + b] = iface ? P->gamma * (I - nn) * gn : 0.0;",
                                "st->Pi[3 * a + b] = iface ? 0.8 * P->gamma * (I - nn) * gn : 0.0;"),
    "wall volume doubled": ("return P->dim == 2 ? P->dx * P->dx : P->dx * P->dx * P->dx;",
                            "return P->dim == 2 ? 2.0 * P->dx * P->dx : 2.0 * P->dx * P->dx * P->dx;"),
}


def run_pins_on(source: str, tmp_path):
    mutant_src = tmp_path / "copy.c"
    mutant_src.write_text(source)
    lib = tmp_path / "libcopy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    str(mutant_src), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, SPH_ORACLE_LIB=str(lib))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           *[os.path.join(ROOT, "tests", f) for f in PINS]],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes(tmp_path):
    r = run_pins_on(open(SRC).read(), tmp_path)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    good, bad = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(good) == 1, name
    r = run_pins_on(src.replace(good, bad), tmp_path)
    assert r.returncode != 0, f"no pin caught: {name}\n{r.stdout[-2000:]}"
