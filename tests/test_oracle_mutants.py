"""The pins catch plausible mistakes: each case plants one mistake in a copy
of the oracle (on the CPU), builds it, runs the pin tests against it in a
child process and requires that at least one pin fails.

Planted mistakes: the chemical-potential sign as printed in
eq:chemical_potential, a c_s^2 slip in eq:gradient_phi, a transposed velocity
component, a missing 1/c_s^2 in eq:force_term, a flipped pressure force
(eq:pressure_force), a flipped viscous force (eq:viscous_force_wmrt), the
wrong stress row relaxed at s_nu, bounce-back into the wrong slot
(eq:no_slip_f), the inlet's tangential factor N = 4 as printed, a missing
1/2 in the g equilibrium shift (eq:equilibrium_with_force), the velocity
inlet applied to f instead of f' = f + F/2 (eq:velocity_boundary_u), and three
outlet mistakes (eq:implicit_convective): the old and new layers swapped, the
outlet speed not clamped to [0, 1], and the speed taken on layer N instead of
N-1.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")

FAST = ["tests/test_oracle_lattice.py", "tests/test_oracle_faces.py", "tests/test_oracle_physics.py",
        "-m", "not slow"]
ALL = ["tests/test_oracle_lattice.py", "tests/test_oracle_faces.py", "tests/test_oracle_physics.py"]

MUTANTS = {
    "mu_phi_printed_sign": (
        "double mu_phi = 4.0 * beta * (phi - 0.0) * (phi - 1.0) * (phi - 0.5) - kappa * lap;",
        "double mu_phi = 4.0 * beta * phi * (1.0 - phi) * (phi - 0.5) - kappa * lap;", FAST),
    "gradient_cs2_slip": (
        "gphi[d] += c->e[a][d] * c->w[a] * phin[a] / CS2;",
        "gphi[d] += c->e[a][d] * c->w[a] * phin[a] / 0.5;", FAST),
    "transposed_velocity": (
        "for (int d = 0; d < 3; ++d) c->e[a][d] = M_D3Q19[1 + d][a];",
        "for (int d = 0; d < 3; ++d) c->e[a][d] = M_D3Q19[1 + (d + 1) % 3][a];", FAST),
    "force_term_missing_cs2": (
        "Fa[a] = c->w[a] * eF / (rho * CS2);",
        "Fa[a] = c->w[a] * eF / rho;", FAST),
    "pressure_force_sign": (
        "Fp[d] = -pstar * CS2 * gr[d];",
        "Fp[d] = pstar * CS2 * gr[d];", ALL),
    "viscous_force_sign": (
        "Fmu[i] = -nu / CS2 * acc;",
        "Fmu[i] = nu / CS2 * acc;", ALL),
    "wrong_stress_row": (
        "for (int k = 4; k <= 8; ++k) c->shear[k] = 1;  /* eq:23 */",
        "for (int k = 5; k <= 9; ++k) c->shear[k] = 1;  /* eq:23 */", FAST),
    "bounce_back_slot": (
        "c->fB[i * Q + a] = c->fs[i * Q + c->opp[a]];",
        "c->fB[i * Q + a] = c->fs[i * Q + a];", ALL),
    "inlet_factor_quarter": (
        "double fpa = fp[ab] + (Ga - Gab) - 0.5 * eM;",
        "double fpa = fp[ab] + (Ga - Gab) - 0.25 * eM;", FAST),
    "inlet_missing_force_shift": (
        "half[a] = 0.5 * c->w[a] * eF / (rho * CS2);",
        "half[a] = 0.0;", FAST),
    "outlet_swapped_layers": (
        "fB[iN * Q + a] = (fA[iN * Q + a] + lam * fB[iM * Q + a]) / (1.0 + lam);",
        "fB[iN * Q + a] = (fB[iM * Q + a] + lam * fA[iN * Q + a]) / (1.0 + lam);", FAST),
    "outlet_unclamped": (
        "double lam = U < 0.0 ? 0.0 : (U > 1.0 ? 1.0 : U);",
        "double lam = U;", FAST),
    "outlet_speed_wrong_layer": (
        "int64_t iM = (c->D == 2) ? nid(c, t0, nL - 2, 0) : nid(c, t0, t1, nL - 2);",
        "int64_t iM = (c->D == 2) ? nid(c, t0, nL - 1, 0) : nid(c, t0, t1, nL - 1);", FAST),
    "g_shift_missing_half": (
        "double gbar = geq - 0.5 * Fphi;",
        "double gbar = geq - Fphi;", ALL),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    from oracle import oracle
    old, new, selection = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: %s" % name
    mutant = tmp_path / "lbm_oracle_mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mutant), str(tmp_path / "liblbm_oracle_mutant.so"))
    env = dict(os.environ, LBM_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + selection,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, "no pin failed for %s:\n%s" % (name, r.stdout[-2000:])
