"""The oracle's pins catch plausible mistakes.

Each case plants one plausible mistake (a dropped term, a wrong sign, a
swapped index or operand) in a copy of the oracle's C source - never in the
oracle itself; in every place the rule is written, for the integer raster
rules the two visibility forms share - builds the copy, points the oracle's loader at it and runs
the pins of tests/test_oracle_pins.py that cover that part.  The case passes
when the pin named for it fails on the mutant.  The BRDF terms have their
own cases in test_oracle_pins.py.  No GPU is used.
"""
import ctypes
import inspect
import subprocess

import pytest

import test_oracle_pins as PINS
from oracle import oracle as O
from paper_2407_10707_gb300 import synth

SKIN_PINS = ("test_fk_identity_pose_gives_identity_bones", "test_fk_root_rotation_is_rigid",
             "test_fk_chain_closed_form", "test_fk_chain_noncommuting_rotations",
             "test_skin_eq1_inverse_distance_weights", "test_skin_covariance_of_a_known_rotation",
             "test_skin_displacement_moves_vertices_and_gaussians", "test_skin_identity_pose",
             "test_skin_rigid_motion", "test_skin_eq1_on_a_vertex_and_equidistant",
             "test_skin_normals_under_a_blended_pose")
VIS_PINS = ("test_visibility_single_triangle_visible_from_both_sides", "test_visibility_parallel_quads_occlusion",
            "test_visibility_convex_sphere_hemisphere", "test_visibility_depth_map_of_a_plane",
            "test_visibility_covers_exactly_the_pixel_centres_inside")
SHADE_PINS = ("test_shade_lambertian_constant_light_all_visible", "test_shade_visibility_is_linear_in_the_bits",
              "test_shade_light_reads_the_bit_of_its_viewpoint", "test_shade_normal_incidence_closed_form",
              "test_shade_sums_the_pinned_brdf_terms", "test_shade_backface_cull")
PROJECT_PINS = ("test_project_isotropic_on_axis_closed_form", "test_project_offaxis_matches_numeric_jacobian",
                "test_project_validity_rules", "test_project_rect_contains_the_alpha_support")
COMPOSITE_PINS = ("test_composite_one_and_two_gaussians_closed_form", "test_composite_alpha_is_clamped_at_0_99",
                  "test_composite_weights_sum_to_at_most_one_and_stop_rule")
BIN_PINS = ("test_bin_matches_pairwise_enumeration",)

# (id, source text, planted text, pins to run, pin that must fail)
MUTATIONS = [
    # forward kinematics and skinning (Sec. 3.1, Eq. 1)
    ("fk_child_before_parent", "mat3_mul(Rg + 9 * p, Rl, Rg + 9 * j);", "mat3_mul(Rl, Rg + 9 * p, Rg + 9 * j);",
     SKIN_PINS, "test_fk_chain_noncommuting_rotations"),
    ("fk_rest_offset_dropped", "bone[12 * j + 4 * i + 3] = tg[3 * j + i] - rj[i];",
     "bone[12 * j + 4 * i + 3] = tg[3 * j + i];", SKIN_PINS, "test_fk_identity_pose_gives_identity_bones"),
    ("rodrigues_transposed", "double K[9] = {0, -r[2], r[1], r[2], 0, -r[0], -r[1], r[0], 0};",
     "double K[9] = {0, r[2], -r[1], -r[2], 0, r[0], r[1], -r[0], 0};", SKIN_PINS,
     "test_fk_root_rotation_is_rigid"),
    ("eq1_inverse_square", "u[j] = 1.0 / (d > 1e-8 ? d : 1e-8);",
     "u[j] = 1.0 / ((d > 1e-8 ? d : 1e-8) * (d > 1e-8 ? d : 1e-8));", SKIN_PINS,
     "test_skin_eq1_inverse_distance_weights"),
    ("eq1_not_normalised", "for (int j = 0; j < K; ++j) u[j] /= usum;", "for (int j = 0; j < K; ++j) u[j] *= 1.0;",
     SKIN_PINS, "test_skin_identity_pose"),
    ("quaternion_conjugated", "double qw = q[0] / qn,", "double qw = -q[0] / qn,", SKIN_PINS,
     "test_skin_covariance_of_a_known_rotation"),
    ("scale_not_squared", "s2[i] = exp(2.0 * logscale[3 * g + i]);", "s2[i] = exp(logscale[3 * g + i]);",
     SKIN_PINS, "test_skin_identity_pose"),
    ("covariance_right_factor_untransposed", "for (int k = 0; k < 3; ++k) t += MS[3 * i + k] * M[3 * j + k];",
     "for (int k = 0; k < 3; ++k) t += MS[3 * i + k] * M[3 * k + j];", SKIN_PINS, "test_skin_rigid_motion"),
    ("gaussian_displacement_dropped", "double xb[3] = {x[0] + dx[0], x[1] + dx[1], x[2] + dx[2]};",
     "double xb[3] = {x[0], x[1], x[2]};", SKIN_PINS, "test_skin_displacement_moves_vertices_and_gaussians"),
    ("vertex_displacement_dropped", "x[i] = xv[3 * v + i] + (dxv ? dxv[3 * v + i] : 0.0);",
     "x[i] = xv[3 * v + i];", SKIN_PINS, "test_skin_displacement_moves_vertices_and_gaussians"),
    ("normal_not_renormalised", "nd[3 * g + i] = m[i] / ml;", "nd[3 * g + i] = m[i];", SKIN_PINS,
     "test_skin_normals_under_a_blended_pose"),
    # visibility (Sec. 3.2, depth-map form)
    ("depth_bias_subtracted", "(Z[v] <= depth[pix] + biasq)", "(Z[v] <= depth[pix] - biasq)", VIS_PINS,
     "test_visibility_single_triangle_visible_from_both_sides"),
    ("depth_sign_flipped", "Z[v] = floor_div(-z, 1024);", "Z[v] = floor_div(z, 1024);", VIS_PINS,
     "test_visibility_parallel_quads_occlusion"),
    ("edge_function_dropped", "if (wa < 0 || wb < 0 || wc < 0) continue;", "if (wa < 0 || wb < 0) continue;",
     VIS_PINS, "test_visibility_covers_exactly_the_pixel_centres_inside"),
    ("depth_weights_swapped", "floor_div(wa * Z[a] + wb * Z[b] + wc * Z[c], area);",
     "floor_div(wa * Z[a] + wb * Z[c] + wc * Z[b], area);", VIS_PINS, "test_visibility_depth_map_of_a_plane"),
    # shading (Eq. 2)
    ("cosine_dropped", "* light_A[k] * vis * ci * (ag[3 * g + c] / ORC_PI + p * fsp);",
     "* light_A[k] * vis * (ag[3 * g + c] / ORC_PI + p * fsp);", SHADE_PINS,
     "test_shade_lambertian_constant_light_all_visible"),
    ("diffuse_without_pi", "* light_A[k] * vis * ci * (ag[3 * g + c] / ORC_PI + p * fsp);",
     "* light_A[k] * vis * ci * (ag[3 * g + c] + p * fsp);", SHADE_PINS,
     "test_shade_lambertian_constant_light_all_visible"),
    ("below_horizon_lights_kept", "if (!(ci > 0.0)) continue;", "if (ci == 0.0) continue;", SHADE_PINS,
     "test_shade_lambertian_constant_light_all_visible"),
    ("gamma_inverted", "pow(Lo[c] > 1e-6 ? Lo[c] : 1e-6, 1.0 / 2.2);", "pow(Lo[c] > 1e-6 ? Lo[c] : 1e-6, 2.2);",
     SHADE_PINS, "test_shade_lambertian_constant_light_all_visible"),
    ("light_ignores_its_viewpoint", "int d = dmap[k];", "int d = k;", SHADE_PINS,
     "test_shade_light_reads_the_bit_of_its_viewpoint"),
    ("visibility_word_index_dropped", "uint32_t word = bits[(size_t)v * DW + (d >> 5)];",
     "uint32_t word = bits[(size_t)v * DW];", SHADE_PINS, "test_shade_light_reads_the_bit_of_its_viewpoint"),
    ("half_vector_difference", "double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};",
     "double h[3] = {wi[0] - wo[0], wi[1] - wo[1], wi[2] - wo[2]};", SHADE_PINS,
     "test_shade_normal_incidence_closed_form"),
    ("view_vector_reversed", "double wo[3] = {cam_center[0] - x[0], cam_center[1] - x[1], cam_center[2] - x[2]};",
     "double wo[3] = {x[0] - cam_center[0], x[1] - cam_center[1], x[2] - cam_center[2]};", SHADE_PINS,
     "test_shade_sums_the_pinned_brdf_terms"),
    # EWA projection (3DGS conventions)
    ("low_pass_dropped", "double s00 = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + 0.3;",
     "double s00 = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2];", PROJECT_PINS,
     "test_project_isotropic_on_axis_closed_form"),
    ("jacobian_sign", "-fx * p[0] / (z * z)", "fx * p[0] / (z * z)", PROJECT_PINS,
     "test_project_offaxis_matches_numeric_jacobian"),
    ("conic_offdiagonal_sign", "conic[3 * g + 1] = -s01 / det;", "conic[3 * g + 1] = s01 / det;", PROJECT_PINS,
     "test_project_offaxis_matches_numeric_jacobian"),
    ("support_radius_halved", "double r2 = 2.0 * log(255.0 * o);", "double r2 = log(255.0 * o);", PROJECT_PINS,
     "test_project_rect_contains_the_alpha_support"),
    ("near_plane_dropped", "p[2] > 0.2 && o > 1.0 / 255.0", "p[2] > 0.0 && o > 1.0 / 255.0", PROJECT_PINS,
     "test_project_validity_rules"),
    # compositing (3DGS blending)
    ("alpha_unclamped", "double a = araw < 0.99 ? araw : 0.99;", "double a = araw;", COMPOSITE_PINS,
     "test_composite_alpha_is_clamped_at_0_99"),
    ("transmittance_dropped", "C[c] += color[3 * g + c] * a * T;", "C[c] += color[3 * g + c] * a;",
     COMPOSITE_PINS, "test_composite_one_and_two_gaussians_closed_form"),
    ("back_to_front", "if (x->depth < y->depth) return -1;\n    if (x->depth > y->depth) return 1;",
     "if (x->depth > y->depth) return -1;\n    if (x->depth < y->depth) return 1;", COMPOSITE_PINS,
     "test_composite_one_and_two_gaussians_closed_form"),
    ("conic_cross_term_halved", "2.0 * conic[3 * g + 1] * dx * dy", "conic[3 * g + 1] * dx * dy",
     COMPOSITE_PINS, "test_composite_one_and_two_gaussians_closed_form"),
    ("stop_threshold", "if (test < 1e-4) break;", "if (test < 1e-3) break;", COMPOSITE_PINS,
     "test_composite_weights_sum_to_at_most_one_and_stop_rule"),
    # binning
    ("last_tile_column_dropped", "r[0] / TS <= cx && cx <= r[2] / TS", "r[0] / TS <= cx && cx < r[2] / TS",
     BIN_PINS, "test_bin_matches_pairwise_enumeration"),
    ("depth_ties_by_descending_index", "return (x->idx > y->idx) - (x->idx < y->idx);\n}\n\nlong orc_bin",
     "return (x->idx < y->idx) - (x->idx > y->idx);\n}\n\nlong orc_bin", BIN_PINS,
     "test_bin_matches_pairwise_enumeration"),
]


def _run_pin(name):
    fn = getattr(PINS, name)
    kwargs = {}
    if "small_avatar" in inspect.signature(fn).parameters:
        kwargs["small_avatar"] = synth.make_avatar(642, 300, seed=5)
    fn(**kwargs)


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_planted_mistake(case, tmp_path, monkeypatch):
    mid, old, new, pins, expect = case
    assert expect in pins
    src = open(O._SRC).read()
    assert src.count(old) >= 1, f"{mid}: the source text to mutate is missing"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))   # every copy of a shared rule (the two visibility forms)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                           str(path), "-lm"])
    monkeypatch.setattr(O, "_LIB_PATH", str(so))
    monkeypatch.setattr(O, "_lib", None)
    assert isinstance(O.lib(), ctypes.CDLL)
    failed = []
    for name in pins:
        try:
            _run_pin(name)
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
            failed.append(name)
    assert expect in failed, f"{mid}: {expect} passes the planted mistake (pins that failed: {failed})"


def test_every_unmutated_pin_passes_through_the_same_loader(tmp_path, monkeypatch):
    """The harness itself: the unchanged source built the same way passes
    every pin the mutation cases run."""
    so = tmp_path / "libsame.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                           O._SRC, "-lm"])
    monkeypatch.setattr(O, "_LIB_PATH", str(so))
    monkeypatch.setattr(O, "_lib", None)
    for name in sorted({p for m in MUTATIONS for p in m[3]}):
        _run_pin(name)
