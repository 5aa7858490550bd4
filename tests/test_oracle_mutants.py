"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a temporary copy of the oracle source
(on the CPU, never in the committed oracle), builds it, points the oracle's
Python front end at the mutant and runs the pin tests of test_oracle_pins.py.
At least one pin must fail for every mutant; the unmodified oracle passes them
all (that is test_oracle_pins.py itself).
"""
import os
import shutil
import subprocess

import pytest

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ORC = os.path.join(os.path.dirname(HERE), "oracle")

# (name, original text, planted mistake)
MUTANTS = [
    ("shear wave dropped", "diss = diss + l2 * beta[i] * ri;", "diss = diss;"),
    ("acoustic strength sign", "T alpha1 = (dp - rho_t * c_t * du[d])", "T alpha1 = (dp + rho_t * c_t * du[d])"),
    ("Roe weights swapped", "u_t[i] = (sL * uL[i] + sR * uR[i]) / (sL + sR);",
     "u_t[i] = (sR * uL[i] + sL * uR[i]) / (sL + sR);"),
    ("entropy-fix denominator", "return (lambda * lambda + delta * delta) / (2.0 * delta);",
     "return (lambda * lambda + delta * delta) / delta;"),
    ("energy flux without pressure", "F[nv - 1] = (Q[nv - 1] + p) * vn;", "F[nv - 1] = Q[nv - 1] * vn;"),
    ("momentum flux index", "F[1 + i] = rho * u[i] * vn", "F[1 + i] = rho * u[d] * vn"),
    ("minmod picks the larger slope", "if (value(a) > 0.0 && value(b) > 0.0) return value(a) < value(b) ? a : b;",
     "if (value(a) > 0.0 && value(b) > 0.0) return value(a) < value(b) ? b : a;"),
    ("MUSCL right state sign", "QR = q2 - e4 * sumR;", "QR = q2 + e4 * sumR;"),
    ("periodic ghost on the low side", "if (c < 0) return bc[0] == BC_PERIODIC ? ((c % n) + n) % n : 0;",
     "if (c < 0) return bc[0] == BC_PERIODIC ? 0 : 0;"),
    ("residual sign", "R[(size_t)v * ncell + cidx] += (Fh - Fl) * ds;", "R[(size_t)v * ncell + cidx] += (Fl - Fh) * ds;"),
    ("face area of the wrong axis", "if (a != d) ds *= L.h[a];\n    int e[3]", "if (a == d) ds *= L.h[a];\n    int e[3]"),
    ("RK stage 2 weights", "U2[c] = 0.75 * U[c] + 0.25 * (", "U2[c] = 0.5 * U[c] + 0.5 * ("),
    ("RK stage 3 weights", "U[c] = (1.0 / 3.0) * U[c] + (2.0 / 3.0) * (", "U[c] = 0.5 * U[c] + 0.5 * ("),
    ("CFL wave speed", "sum = sum + (fabs(u[a]) + c) / L.h[a];", "sum = sum + (fabs(u[a]) - c) / L.h[a];"),
    ("sampled residual: stencil shifted by one cell", "c3[d] += side + t - 2;", "c3[d] += side + t - 1;"),
    ("sampled residual: boundary of the wrong axis", "const int sj = ghost_source(c3[1], L.n[1], g.bc[1]);",
     "const int sj = ghost_source(c3[1], L.n[1], g.bc[0]);"),
    ("sampled residual: source sign", "R[v] = R[v] - vol * T(S[(size_t)v * L.cells() + (size_t)id]);",
     "R[v] = R[v] + vol * T(S[(size_t)v * L.cells() + (size_t)id]);"),
]


def _pin_checks():
    import test_oracle_cells as C
    import test_oracle_pins as P
    return [
        lambda: P.test_free_stream_residual_is_exactly_zero(2, 0),
        lambda: P.test_free_stream_residual_is_exactly_zero(3, 1),
        lambda: P.test_periodic_residual_sums_to_zero_and_rk_conserves(2),
        lambda: P.test_textbook_jacobian_matches_finite_differences_of_the_flux(2, 0),
        lambda: P.test_textbook_jacobian_matches_finite_differences_of_the_flux(3, 2),
        lambda: P.test_roe_flux_equals_half_sum_minus_abs_roe_matrix_jump(2),
        lambda: P.test_roe_flux_equals_half_sum_minus_abs_roe_matrix_jump(3),
        P.test_roe_flux_of_equal_states_is_the_physical_flux_bitwise,
        P.test_supersonic_roe_flux_is_upwind,
        P.test_entropy_fix_only_acts_near_sonic_points,
        P.test_entropy_fix_is_continuous_at_its_threshold,
        P.test_muscl_is_exact_on_linear_data_and_kappa_free_with_minmod,
        P.test_transpose_symmetry_2d_bitwise,
        P.test_rotation_by_90_degrees_2d,
        P.test_periodic_translation_invariance_bitwise,
        P.test_3d_with_uniform_z_reduces_to_2d,
        P.test_time_step_of_uniform_flow_closed_form,
        P.test_ssp_rk3_is_third_order_in_time,
        lambda: P.test_sod_tube_converges_to_exact_solution(0),
        lambda: C.test_residual_cells_equal_the_full_residual_bitwise("2d_6x5_mixed", "minmod", True),
        lambda: C.test_residual_cells_equal_the_full_residual_bitwise("3d_5x6x7_mixed", "primitive", False),
    ]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = open(os.path.join(ORC, "fv_oracle.hpp")).read()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    (tmp_path / "fv_oracle.hpp").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ORC, "fv_oracle.cpp"), tmp_path / "fv_oracle.cpp")
    so = str(tmp_path / "libmutant.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", so,
                    str(tmp_path / "fv_oracle.cpp")], check=True)
    saved = O._lib
    O._lib = O.load_library(so)
    caught = []
    try:
        for chk in _pin_checks():
            try:
                chk()
            except Exception as e:  # an assertion, or a non-physical state the mistake produced
                caught.append(type(e).__name__)
                break
    finally:
        O._lib = saved
    assert caught, f"no pin caught the planted mistake: {name}"
