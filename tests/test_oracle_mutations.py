"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU), rebuilds it,
and checks that at least one pin of test_oracle_pins fails against it."""
import pytest

import oracle
from tests import test_oracle_pins as pins
from tests import test_oracle_terms as term_pins

MUTATIONS = {
    "inverse_transposed": ("inv[3 * i + j] = C[3 * j + i] / det;", "inv[3 * i + j] = C[3 * i + j] / det;"),
    "dv_vd_swapped": ("int d1 = (t == 1 || t == 3), d2 = (t == 2 || t == 3);",
                      "int d1 = (t == 2 || t == 3), d2 = (t == 1 || t == 3);"),
    "scalar_axis_swapped": ("sin(M_PI * (u + p[1]))", "sin(M_PI * (v + p[1]))"),
    "bulge_jacobian_dropped": ("J[3 * i + j] += bulge[0] * bulge[1 + i] * dbeta[j];", ";"),
    "weight_sign": ("2.0 / ((1.0 - z * z) * dP[G] * dP[G])", "2.0 / ((1.0 + z * z) * dP[G] * dP[G])"),
    "legendre_derivative_sign": ("dP[j] = j * (P[j - 1] - x * P[j]) / (1.0 - x * x);",
                                 "dP[j] = j * (x * P[j] - P[j - 1]) / (1.0 - x * x);"),
    "row_index_order": ("int m1 = r / (Nv_i * Nw_i), n1 = (r / Nw_i) % Nv_i, p1 = r % Nw_i;",
                        "int m1 = r / (Nv_i * Nw_i), p1 = (r / Nw_i) % Nv_i, n1 = r % Nw_i;"),
    "eps_cos": ("double eps = 1.0 + p[0] * sin(kx);", "double eps = 1.0 + p[0] * cos(kx);"),
    "det_sign": ("double det = J[0] * C[0] + J[1] * C[1] + J[2] * C[2];",
                 "double det = J[0] * C[0] - J[1] * C[1] + J[2] * C[2];"),
    "recurrence_term": ("P[j + 1] = ((2.0 * j + 1.0) * x * P[j] - j * P[j - 1]) / (j + 1.0);",
                        "P[j + 1] = ((2.0 * j + 1.0) * x * P[j] + j * P[j - 1]) / (j + 1.0);"),
    "trilinear_shape_sign": ("double s[3] = {(n & 1) ? 1.0 : -1.0,", "double s[3] = {(n & 1) ? -1.0 : 1.0,"),
    "projection_norm": ("C[k] = (2.0 * k + 1.0) / 2.0 * (acc.s + acc.c);", "C[k] = (2.0 * k + 1.0) * (acc.s + acc.c);"),
    # the term-list fill
    "term_block_filter": ("if (tm[0] != gi || tm[1] != gj) continue;", "if (tm[0] != gi) continue;"),
    "term_scale_dropped": ("acc_add(&acc, oj->scales[k] * (", "acc_add(&acc, 1.0 * ("),
    "term_alpha_entry": ("+ sa * na + sb];", "+ sa * na + sa];"),
    "term_row_index": ("int n1 = (r / Nw_i) % Nv_i;\n    int p1 = r % Nw_i;", "int p1 = (r / Nw_i) % Nv_i;\n    int n1 = r % Nw_i;"),
    "term_test_trial_w": ("double fw = fac(ch, tm[6], p1, c) * fac(ch, tm[9], p2, c);",
                          "double fw = fac(ch, tm[9], p1, c) * fac(ch, tm[6], p2, c);"),
}

PIN_CALLS = [
    lambda: pins.test_gauss_legendre_matches_numpy(8),
    lambda: pins.test_legendre_values_and_derivatives_match_numpy(),
    lambda: [pins.test_linearisation_projection_matches_adams_neumann(t) for t in pins.TYPES],
    lambda: pins.test_unit_alpha_scalar_closed_form(3, 3),
    lambda: pins.test_unit_cube_metric_is_half_identity(),
    lambda: pins.test_polynomial_alpha_is_integrated_exactly(3),
    lambda: pins.test_scalar_alpha_axes_against_adaptive_quadrature(),
    lambda: pins.test_geometry_map_corners_centre_and_jacobian(),
    lambda: pins.test_metric_coupling_defining_identity(),
    lambda: pins.test_direct_equals_product_to_sum_small_orders("metric"),
    lambda: pins.test_invariants_on_curved_metric_element(),
    lambda: term_pins.test_diffusion_on_unit_cube_closed_form(),
    lambda: term_pins.test_random_terms_match_brute_force_metric(),
    lambda: term_pins.test_random_terms_match_brute_force_scalar(),
]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source()
    assert src.count(old) == 1, "mutation anchor not found exactly once: %s" % name
    path = oracle.build_variant(src.replace(old, new), str(tmp_path / ("or_%s.so" % name)))
    caught = []
    with oracle.use_library(path):
        for call in PIN_CALLS:
            try:
                call()
            except (AssertionError, RuntimeError, ValueError, FloatingPointError):
                caught.append(call)
    assert caught, "no pin caught mutation %s" % name
