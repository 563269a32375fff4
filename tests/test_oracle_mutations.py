"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each mutation edits one expression of ``ddgi_oracle.c`` (a dropped term, a
wrong sign, a transposed index, a swapped operand), compiles the copy, routes
the oracle wrappers through it and runs the pin battery: at least one pin
must fail.  This guards the pins themselves against being too weak.
"""
import os

import pytest

import oracle
import test_oracle_converge as conv
import test_oracle_pins as pins
import test_oracle_texel_grad as tgrad

BATTERY = [
    lambda: pins.test_spherical_fibonacci_structure(64),
    pins.test_frame_dirs_are_rotated_sf,
    pins.test_oct_axes_closed_form,
    pins.test_oct_round_trips,
    lambda: pins.test_bilinear_reproduces_affine_tile(6),
    lambda: pins.test_border_copy_makes_sampling_continuous_across_seams(6),
    pins.test_trace_matches_exact_rational_brute_force,
    pins.test_enclosing_box_distances_closed_form,
    lambda: pins.test_uniform_sky_gives_exact_mean(64),
    pins.test_linear_sky_converges_to_cosine_mean,
    pins.test_hysteresis_gamma_closed_forms,
    pins.test_furnace_multibounce_exact,
    pins.test_direct_light_and_sky_per_ray,
    pins.test_shadow_ray_blocks_sun,
    pins.test_query_agreeing_probes_return_common_value,
    pins.test_query_chebyshev_and_backface_weights_by_hand,
    pins.test_query_at_a_probe_uses_only_that_probe,
    pins.test_self_shadow_bias_moves_the_sample_point,
    pins.test_states_hand_built,
    pins.test_states_backface_fraction_threshold,
    pins.test_cascade_weights_nested,
    conv.test_converge_uniform_sky_exact_and_states,
    conv.test_converge_batches_are_distinct_rotations,
    conv.test_converge_enclosing_sphere_moments,
    lambda: tgrad.test_texel_gradient_matches_central_differences(5.0),
    tgrad.test_texel_gradient_fold_is_the_interior_gradient,
]

MUTATIONS = {
    "blend_unnormalised": ("enew[k] = pow(m[k] / sw, 1.0 / v->gamma);", "enew[k] = pow(m[k], 1.0 / v->gamma);"),
    "bias_sign": ("    for (int a = 0; a < 3; ++a)\n        xb[a] = x[a] + (0.2 * n[a] + 0.8 * wo[a])",
                  "    for (int a = 0; a < 3; ++a)\n        xb[a] = x[a] + (0.2 * n[a] - 0.8 * wo[a])"),
    "border_unmirrored": ("TILE(tile, N, C, 0,     k)[c] = TILE(tile, N, C, 1, n + 1 - k)[c];",
                          "TILE(tile, N, C, 0,     k)[c] = TILE(tile, N, C, 1, k)[c];"),
    "bilinear_transposed": ("double tx = sx - (double)x0, ty = sy - (double)y0;\n    for (int64_t c = 0;",
                            "double ty = sx - (double)x0, tx = sy - (double)y0;\n    for (int64_t c = 0;"),
    "backface_depth": ("out[3] = fmin(0.2 * t, v->t_max);", "out[3] = fmin(t, v->t_max);"),
    "chebyshev_square": ("wc = var / (var + dr * dr);", "wc = var / (var + dr);"),
    "gamma_decode": ("pow(fmax(e[k], 0.0), 0.5 * v->gamma)", "pow(fmax(e[k], 0.0), v->gamma)"),
    "threshold_order": ("if (delta > v->thr_high) a = 0.0;", "if (delta > v->thr_high) a = a;"),
    "sf_offset": ("double z = 1.0 - (2.0 * (double)i + 1.0) / (double)n;",
                  "double z = 1.0 - (2.0 * (double)i) / (double)n;"),
    "trilinear_flipped": ("for (int a = 0; a < 3; ++a) wt *= o[a] ? fr[a] : 1.0 - fr[a];",
                          "for (int a = 0; a < 3; ++a) wt *= o[a] ? 1.0 - fr[a] : fr[a];"),
    "direct_no_pi": ("direct[k] = L->sun_irradiance[k] * cosl / M_PI;\n    }\n    /* indirect",
                     "direct[k] = L->sun_irradiance[k] * cosl;\n    }\n    /* indirect"),
    "lerp_swapped": ("for (int k = 0; k < 3; ++k) old[k] = (1.0 - a) * enew[k] + a * old[k];",
                     "for (int k = 0; k < 3; ++k) old[k] = a * enew[k] + (1.0 - a) * old[k];"),
    "indirect_dropped": ("out[k] = Le[k] + rho[k] * (direct[k] + M[k]);", "out[k] = Le[k] + rho[k] * direct[k];"),
    "state_threshold": ("if (4 * bf > R) st = OR_OFF;", "if (2 * bf > R) st = OR_OFF;"),
    "oct_lower_fold": ("double qx = (1.0 - fabs(py)) * signnz(px);", "double qx = (1.0 - fabs(px)) * signnz(px);"),
    "cascade_falloff": ("w *= clampd(m, 0.0, 1.0);", "w *= clampd(m + 1.0, 0.0, 1.0);"),
    "distance_square_moment": ("mu2 += w * dd * dd;", "mu2 += w * dd;"),
    "tie_break": ("if (tri_intersect(s, k, o, d, &tk, &bk) && tk < best)",
                  "if (tri_intersect(s, k, o, d, &tk, &bk) && tk > 0.0 && (bi < 0 || tk > best))"),
    "converge_one_rotation": ("0xD1B54A32D192ED03ULL * (uint64_t)(b + 1)", "0xD1B54A32D192ED03ULL * (uint64_t)1"),
    "converge_unencoded": ("e[k] = pow(num_i[4 * t + k] / num_i[4 * t + 3], 1.0 / v->gamma);",
                           "e[k] = num_i[4 * t + k] / num_i[4 * t + 3];"),
    "converge_no_advance": ("states[p] = advanced(states[p]);", "(void)0;"),
    "texel_grad_gamma_chain": ("double db = da * 0.5 * v->gamma * pow(b[k], 0.5 * v->gamma - 1.0);",
                               "double db = da * 0.5 * v->gamma;"),
    "texel_grad_bilinear_swapped": ("g_irr[p * tsi + (by[j] * N + bx[j]) * 3 + k] += db * bw[j];",
                                    "g_irr[p * tsi + (by[j] * N + bx[j]) * 3 + k] += db * bw[3 - j];"),
    "texel_grad_fold_corner": ("TILE(g_tile, N, C, n, n)[c] += TILE(g_tile, N, C, 0, 0)[c];",
                               "TILE(g_tile, N, C, 1, 1)[c] += TILE(g_tile, N, C, 0, 0)[c];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    handle = oracle.build_variant(str(path), str(tmp_path / f"libmutant_{os.getpid()}.so"))
    failures = 0
    with oracle.use_library(handle):
        for check in BATTERY:
            try:
                check()
            except AssertionError:
                failures += 1
    assert failures >= 1, f"no pin caught mutation {name}"
