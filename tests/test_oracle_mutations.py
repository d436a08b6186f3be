"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each.

The mutated C source is compiled to a temporary library and the pin module
runs against it in a subprocess (``NB_ORACLE_LIB``). Every mutation must make
at least one pin fail; the unmodified oracle passes them all (see
``test_oracle_pins.py``).
"""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "drop_exp_term_of_coulomb_force": ("2.0 * beta / sqrt(M_PI) * exp(-beta * beta * r2)", "0.0"),
    "reaction_force_wrong_sign": ("Fl[3 * j + k] -= s * d[k];", "Fl[3 * j + k] += s * d[k];"),
    "lj_force_wrong_prefactor": ("12.0 * c12 * rinv6 * rinv6", "6.0 * c12 * rinv6 * rinv6"),
    "missing_lj_potential_shift": (" - (c12 * rc12 - c6 * rc6)", ""),
    "erfc_argument_squared": ("erfc(beta * r) / r", "erfc(beta * r2) / r"),
    "exclusions_ignored": ("if (is_excluded(i, j, excl_off, excl_idx)) continue;\n                    const", "const"),
    "min_image_uses_floor": ("v -= box[k] * rint(v / box[k]);", "v -= box[k] * floor(v / box[k]);"),
    "coulomb_constant_dropped": ("double qq = ORACLE_COULOMB_F * qi * qj;", "double qq = qi * qj;"),
    # the FP32 contract's image of a displaced position (search frame x0 != current frame x)
    "fp32_image_uses_floor": ("float k = rintf((x - w0) / L);", "float k = floorf((x - w0) / L);"),
    "fp32_image_sign_slip": ("return x - k * L;", "return x + k * L;"),
    # the energies at the contract's distances
    "energy_f32_drops_the_shift": ("const float dx = u[0] + (float)sx * box[0];", "const float dx = u[0];"),
    "energy_f32_lj_parameters_swapped": ("q[i], q[j], c[0], c[1], (double)rcf", "q[i], q[j], c[1], c[0], (double)rcf"),
    "energy_f32_shift_at_the_fp64_cutoff": ("c[0], c[1], (double)rcf, beta", "c[0], c[1], rc, beta"),
    "energy_f32_partner_charge": ("pair_terms((double)r2, q[i], q[j],", "pair_terms((double)r2, q[i], q[i],"),
}

# mistakes in the force adjoint, caught by tests/test_oracle_adjoint.py
ADJOINT_MUTATIONS = {
    "adjoint_missing_gaussian_term": (" - 2.0 * K * cb * beta * beta * e * rinv2", ""),
    "adjoint_lj_second_derivative": ("168.0 * c12", "144.0 * c12"),
    "adjoint_charge_uses_own_charge": ("gql[i] += ORACLE_COULOMB_F * q[j] * B * ud;",
                                       "gql[i] += ORACLE_COULOMB_F * q[i] * B * ud;"),
    "adjoint_lj_not_symmetrised": ("gljl[ba] += 0.5 * d6;", ""),
    "adjoint_reaction_sign": ("gxl[3 * j + k] -= v;", "gxl[3 * j + k] += v;"),
}


# mistakes in the Coulomb options (reaction field, shift, exclusion
# correction), caught by tests/test_oracle_coul.py
COUL_MUTATIONS = {
    "rf_quadratic_term_sign": ("*phi = 1.0 / r + k_rf * r2 - c_rf;", "*phi = 1.0 / r - k_rf * r2 - c_rf;"),
    "rf_force_constant_halved": ("*B = rinv2 / r - 2.0 * k_rf;", "*B = rinv2 / r - k_rf;"),
    "rf_conducting_constant": ("*k_rf = 1.0 / (2.0 * rc * rc * rc);", "*k_rf = 1.0 / (rc * rc * rc);"),
    "rf_adjoint_sign": ("*D = -3.0 * rinv2 * rinv2 / r;", "*D = 3.0 * rinv2 * rinv2 / r;"),
    "excluded_energy_sign": ("*phi = -erf(beta * r) / r;", "*phi = erf(beta * r) / r;"),
    "excluded_force_keeps_bare_term": ("*B = Be - rinv2 / r;", "*B = Be;"),
    "ewald_shift_sign": ("*phi = A - shift;", "*phi = A + shift;"),
}

# mistakes in the smooth-PME spread and gather, caught by tests/test_oracle_pme.py
PME_MUTATIONS = {
    "bspline_recursion_denominator": ("(n - u) / (n - 1) * oracle_bspline", "(n - u) / n * oracle_bspline"),
    "bspline_derivative_sign": ("return oracle_bspline(n - 1, u) - oracle_bspline(n - 1, u - 1.0);",
                                "return oracle_bspline(n - 1, u - 1.0) - oracle_bspline(n - 1, u);"),
    "pme_scaled_coordinate_off": ("double u = s * K;", "double u = s * (K - 1);"),
    "spread_grid_index_off_by_one": ("for (int j = 0; j < order; ++j) w[a][j] = oracle_bspline(order, u[a] - (base[a] - j));",
                                     "for (int j = 0; j < order; ++j) w[a][j] = oracle_bspline(order, u[a] - (base[a] - j) + 1.0);"),
    "gather_missing_grid_scale": ("* K[a] / box[a];", ";"),
    "gather_force_sign": ("f[a] -= q[i] * t[a];", "f[a] += q[i] * t[a];"),
    "gather_wrong_axis_derivative": ("w[0][j0] * dw[1][j1] * w[2][j2] * ph", "w[0][j0] * w[1][j1] * dw[2][j2] * ph"),
}

PIN_FILES = {**{k: "test_oracle_pins.py" for k in MUTATIONS},
             **{k: "test_oracle_pme.py" for k in PME_MUTATIONS},
             **{k: "test_oracle_adjoint.py" for k in ADJOINT_MUTATIONS},
             **{k: "test_oracle_coul.py" for k in COUL_MUTATIONS}}


@pytest.mark.parametrize("name", sorted(PIN_FILES))
def test_pins_catch_mutation(name, tmp_path):
    old, new = {**MUTATIONS, **ADJOINT_MUTATIONS, **COUL_MUTATIONS, **PME_MUTATIONS}[name]
    pins = PIN_FILES[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = tmp_path / "oracle_mut.c"
    mutated.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "liboracle_mut.so"))
    env = dict(os.environ, NB_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", pins)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
