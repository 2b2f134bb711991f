"""Planted mistakes in the oracle, each caught by a pin.

Each case copies the oracle and its pins to a scratch directory, changes one
line of the copied nlse_oracle.c (a dropped term, a wrong sign, coefficient
or index, a wrong boundary form), rebuilds it there and runs the pin that must
fail.  A control run of the unchanged copy passes the same pins.  The repo's
own oracle is never touched.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = "tests/test_oracle_pins.py::"

# name: (text in nlse_oracle.c, replacement, pin that must fail)
MUTATIONS = {
    "3d_edge_term_dropped": (
        "sp += PS(0, 1, 1) + PS(0, 1, -1) + PS(0, -1, 1) + PS(0, -1, -1);",
        "sp += PS(0, 1, 1) + PS(0, 1, -1) + PS(0, -1, 1);",
        "test_stationary_dark_soliton_dirichlet[3-2-4-4.0-0.35]"),
    "2d_centre_coefficient": (
        "- 12.0 * DD(0, 0, 0);", "- 11.0 * DD(0, 0, 0);",
        "test_stationary_dark_soliton_dirichlet[2-0-4-4.0-0.35]"),
    "1d_2shoc_coefficient": (
        "(7.0 / 6.0) * DD(0, 0, 0)", "(7.0 / 6.1) * DD(0, 0, 0)",
        "test_bright_soliton_convergence[4-4.0-0.3]"),
    "msd_inward_index": (
        "if (idx[k] == 0) q += g->st[k];", "if (idx[k] == 0) q -= 0;",
        "test_dark_soliton_msd_convergence[2-2.0-0.15]"),
    "msd_ratio_sign": (
        "ratio_re = (D[2 * q] * qr + D[2 * q + 1] * qi) / m2;",
        "ratio_re = (D[2 * q] * qr - D[2 * q + 1] * qi) / m2;",
        "test_dark_soliton_msd_convergence[4-4.0-0.3]"),
    "msd_theta_sign": (
        "theta = (F[2 * q + 1] * qr - F[2 * q] * qi) / m2;",
        "theta = (F[2 * q + 1] * qr + F[2 * q] * qi) / m2;",
        "test_dark_soliton_msd_convergence[2-2.0-0.15]"),
    "dirichlet_Db_sign": (
        "const double f = -(1.0 / g->a) * Nat(g, psi, p);",
        "const double f = (1.0 / g->a) * Nat(g, psi, p);",
        "test_stationary_dark_soliton_dirichlet[1-0-4-4.0-0.35]"),
    "fsplit_V_sign": (
        "F[2 * p] = -g->a * L[2 * p + 1] - g->s * m2 * im + v * im;",
        "F[2 * p] = -g->a * L[2 * p + 1] - g->s * m2 * im - v * im;",
        "test_l0_harmonic_field_in_constant_potential[2-shape0]"),
    "rk4_step8_coefficient": (
        "Ptmp[i] = psi[i] + dt * Ktmp[i];", "Ptmp[i] = psi[i] + half * Ktmp[i];",
        "test_bright_soliton_convergence[2-2.0-0.15]"),
    "rk4_step4_weight": (
        "Ktot[i] = Ktot[i] + 2.0 * Ktmp[i];                          /* 4) */",
        "Ktot[i] = Ktot[i] + 1.0 * Ktmp[i];                          /* 4) */",
        "test_bright_soliton_convergence[2-2.0-0.15]"),
    "energy_nonlinear_sign": (
        "- 0.5 * g.s * m2 * m2", "+ 0.5 * g.s * m2 * m2",
        "test_energy_closed_form[2-shape0-modes0]"),
    "mass_h_power": (
        "*out = pow(h, d) * (acc.sum + acc.c);\n  return 0;\n}\n\nint oracle_energy",
        "*out = pow(h, d - 1) * (acc.sum + acc.c);\n  return 0;\n}\n\nint oracle_energy",
        "test_mass_closed_form_and_exact_sum"),
    "stability_radius": (
        "16.0 * d / (3.0 * h * h)", "16.0 * d / (3.5 * h * h)",
        "test_stability_bound_printed[row1]"),
    "cd_centre_coefficient": (
        "sum += -2.0 * g->d * psi[2 * p + c];", "sum += -2.0 * g->d * psi[2 * p + c] * 1.0000001;",
        "test_bright_soliton_convergence[2-2.0-0.15]"),
    "l0_Fb_dropped": (
        "F[2 * p] = -nb * psi[2 * p + 1];\n      F[2 * p + 1] = nb * psi[2 * p];",
        "F[2 * p] = 0.0;\n      F[2 * p + 1] = 0.0;",
        "test_l0_boundary_sites_follow_their_own_ode[2-shape0]"),
    "l0_Fb_sign": (
        "F[2 * p] = -nb * psi[2 * p + 1];", "F[2 * p] = nb * psi[2 * p + 1];",
        "test_l0_boundary_sites_follow_their_own_ode[2-shape0]"),
    "l0_Nb_at_inward_site": (
        "const double nb = Nat(g, psi, p);", "const double nb = Nat(g, psi, inward(g, p));",
        "test_l0_boundary_sites_follow_their_own_ode[2-shape0]"),
    "l0_Db_dirichlet_form": (
        "} else if (g->bc == BC_L0) {\n      D[2 * p] = 0.0;",
        "} else if (g->bc == BC_L0) {\n      D[2 * p] = -(1.0 / g->a) * Nat(g, psi, p) * re;",
        "test_l0_harmonic_field_in_constant_potential[4-shape0]"),
    "periodic_wrap_modulus": (
        "q += ((idx[k] + o[k] + g->n[k]) % g->n[k]) * g->st[k];",
        "q += ((idx[k] + o[k] + g->n[k]) % (g->n[k] - 1)) * g->st[k];",
        "test_periodic_laplacian_is_its_fourier_symbol[2-shape2]"),
    "periodic_wrap_wrong_axis": (
        "q += ((idx[k] + o[k] + g->n[k]) % g->n[k]) * g->st[k];",
        "q += ((idx[k] + o[0] + g->n[k]) % g->n[k]) * g->st[k];",
        "test_periodic_fourier_modes_exact_rk4[4-shape3-modes3]"),
    "periodic_has_boundary_sites": (
        "  if (g->bc == BC_PERIODIC) return 0;\n", "",
        "test_periodic_laplacian_is_its_fourier_symbol[4-shape3]"),
}


def _copy_tree(dst):
    for sub in ("oracle", "tests", "tests/golden", "paper_1203_1263_gb300"):
        os.makedirs(os.path.join(dst, sub), exist_ok=True)
    for f in ("oracle/__init__.py", "oracle/nlse_oracle.c", "tests/conftest.py", "tests/test_oracle_pins.py",
              "paper_1203_1263_gb300/__init__.py", "paper_1203_1263_gb300/workloads.py"):
        shutil.copy(os.path.join(ROOT, f), os.path.join(dst, f))
    for f in os.listdir(os.path.join(ROOT, "tests", "golden")):
        shutil.copy(os.path.join(ROOT, "tests", "golden", f), os.path.join(dst, "tests", "golden", f))


def _run_pins(dst, pins):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["OMP_NUM_THREADS"] = "2"     # small pins; leaves cores to parallel test workers
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"] + [PINS + p for p in pins],
                          cwd=dst, capture_output=True, text=True, env=env, timeout=600)


def test_unchanged_copy_passes_the_pins(tmp_path):
    _copy_tree(str(tmp_path))
    r = _run_pins(str(tmp_path), sorted({m[2] for m in MUTATIONS.values()}))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_its_pin(name, tmp_path):
    old, new, pin = MUTATIONS[name]
    _copy_tree(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", "nlse_oracle.c")
    text = open(src).read()
    assert text.count(old) == 1, f"the oracle line planted by {name} changed"
    open(src, "w").write(text.replace(old, new))
    r = _run_pins(str(tmp_path), [pin])
    assert r.returncode == 1 and "1 failed" in r.stdout, r.stdout[-2000:]
