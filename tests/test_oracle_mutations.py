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


# ---------------------------------------------------------------- the Python oracles
# (module, id, source text, planted text, pins to run, pin that must fail)
ADJ_PINS = ("test_adjoint_forward_agrees_with_c_oracle", "test_adjoint_matches_central_finite_differences")
SSIM_PINS = ("test_ssim_identity_symmetry_and_constant_images", "test_ssim_of_a_constant_against_a_checkerboard",
             "test_image_loss_weights_and_the_paper_lambda", "test_image_loss_gradient_matches_finite_differences")
REG_PINS = ("test_regularizers_closed_forms", "test_regularizer_weights_are_the_papers",
            "test_regularizer_gradients_match_finite_differences")
MLP_PINS = ("test_mlp_matches_torch_layers_and_closed_forms",)
DENS_PINS = ("test_densify_counts_and_densities", "test_densify_uniform_and_saturated_meshes",
             "test_densify_sampling_follows_the_weights", "test_densify_places_points_uniformly_on_the_triangle")
ADAM_PINS = ("test_adam_matches_torch_and_closed_forms",)

PY_MUTATIONS = [
    ("adjoint", "eq1_inverse_square", "u = 1.0 / torch.clamp(d, min=1e-8)", "u = 1.0 / torch.clamp(d * d, min=1e-8)",
     ADJ_PINS, "test_adjoint_forward_agrees_with_c_oracle"),
    ("adjoint", "specular_without_G1o", "(co[:, None] * (1.0 - kk) + kk))", "1.0)", ADJ_PINS,
     "test_adjoint_forward_agrees_with_c_oracle"),
    ("adjoint", "low_pass_dropped", "s00 = S2[:, 0, 0] + 0.3", "s00 = S2[:, 0, 0]", ADJ_PINS,
     "test_adjoint_forward_agrees_with_c_oracle"),
    ("adjoint", "transmittance_detached", "w = ai * Tex", "w = ai * Tex.detach()", ADJ_PINS,
     "test_adjoint_matches_central_finite_differences"),
    ("adjoint", "gamma_curve_detached", "col = torch.pow(torch.clamp(Lo, min=1e-6), 1.0 / 2.2)",
     "col = torch.pow(torch.clamp(Lo.detach(), min=1e-6), 1.0 / 2.2) + 0.0 * Lo", ADJ_PINS,
     "test_adjoint_matches_central_finite_differences"),
    ("ssim", "c2_tenfold", "C2 = 0.03 ** 2", "C2 = 0.3 ** 2", SSIM_PINS,
     "test_ssim_of_a_constant_against_a_checkerboard"),
    ("ssim", "covariance_without_means", "sxy = _blur(x * y) - mx * my", "sxy = _blur(x * y)", SSIM_PINS,
     "test_ssim_identity_symmetry_and_constant_images"),
    ("ssim", "window_sigma", "SIGMA = 1.5", "SIGMA = 2.5", SSIM_PINS, "test_ssim_identity_symmetry_and_constant_images"),
    ("ssim", "lambda_swapped", "return (1.0 - lam) * l1 + lam * (1.0 - ssim_map(img, target).mean())",
     "return lam * l1 + (1.0 - lam) * (1.0 - ssim_map(img, target).mean())", SSIM_PINS,
     "test_image_loss_weights_and_the_paper_lambda"),
    ("ssim", "torch_loss_halved_dssim", "+ lam * (1.0 - s.mean())", "+ lam * (1.0 - s.mean()) / 2", SSIM_PINS,
     "test_image_loss_gradient_matches_finite_differences"),
    ("regularizers", "smooth_squared", "(av[:, None, :] - av[kv]).abs().sum()", "(av[:, None, :] - av[kv]).pow(2).sum()",
     REG_PINS, "test_regularizers_closed_forms"),
    ("regularizers", "scale_unclamped", "scale = torch.clamp(torch.exp(logscale) - s0, min=0.0).sum()",
     "scale = (torch.exp(logscale) - s0).sum()", REG_PINS, "test_regularizers_closed_forms"),
    ("regularizers", "mdist_squared", "mdist = torch.linalg.vector_norm(xg[:, None, :] - xv[kg], dim=-1).sum()",
     "mdist = ((xg[:, None, :] - xv[kg]) ** 2).sum()", REG_PINS, "test_regularizers_closed_forms"),
    ("regularizers", "smooth_weight", "WEIGHTS = dict(smooth=0.002,", "WEIGHTS = dict(smooth=0.02,", REG_PINS,
     "test_regularizer_weights_are_the_papers"),
    ("mlp", "fourier_without_2pi", "p = 2.0 * np.pi * (", "p = np.pi * (", MLP_PINS,
     "test_mlp_matches_torch_layers_and_closed_forms"),
    ("mlp", "cos_before_sin", "np.concatenate([np.sin(p), np.cos(p)], axis=1)",
     "np.concatenate([np.cos(p), np.sin(p)], axis=1)", MLP_PINS, "test_mlp_matches_torch_layers_and_closed_forms"),
    ("mlp", "last_layer_relu", "return r(h) @ r(W4).T + np.asarray(b4, np.float64)",
     "return np.maximum(r(h) @ r(W4).T + np.asarray(b4, np.float64), 0.0)", MLP_PINS,
     "test_mlp_matches_torch_layers_and_closed_forms"),
    ("densify", "density_over_3kg", "df = S / (6.0 * Kg)", "df = S / (3.0 * Kg)", DENS_PINS,
     "test_densify_counts_and_densities"),
    ("densify", "triangle_search_left", 'i = int(np.searchsorted(cum, s, side="right"))',
     'i = int(np.searchsorted(cum, s, side="left"))', DENS_PINS, "test_densify_sampling_follows_the_weights"),
    ("densify", "no_fold_back", "if u + v > 1.0:", "if u + v > 2.0:", DENS_PINS,
     "test_densify_places_points_uniformly_on_the_triangle"),
    ("adam", "no_bias_correction", "mh = m / (1.0 - b1 ** t)", "mh = m", ADAM_PINS,
     "test_adam_matches_torch_and_closed_forms"),
    ("adam", "second_moment_unsquared", "v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g",
     "v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * np.abs(g)", ADAM_PINS,
     "test_adam_matches_torch_and_closed_forms"),
]


def _mutant_module(modname, old, new):
    import importlib.util
    import types
    spec = importlib.util.find_spec(f"oracle.{modname}")
    src = open(spec.origin).read()
    assert old == "" or src.count(old) == 1, f"{modname}: the source text to mutate is not unique"
    mod = types.ModuleType(f"oracle.{modname}")
    mod.__file__ = spec.origin
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new) if old else src, spec.origin, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("case", PY_MUTATIONS, ids=[f"{m[0]}-{m[1]}" for m in PY_MUTATIONS])
def test_pins_catch_the_planted_mistake_in_the_python_oracles(case, monkeypatch):
    import sys
    import oracle as pkg
    modname, mid, old, new, pins, expect = case
    assert expect in pins
    mut = _mutant_module(modname, old, new)
    monkeypatch.setitem(sys.modules, f"oracle.{modname}", mut)
    monkeypatch.setattr(pkg, modname, mut, raising=False)
    if modname == "adjoint":
        monkeypatch.setattr(PINS, "AJ", mut)
    failed = []
    for name in pins:
        try:
            _run_pin(name)
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError, RuntimeError):
            failed.append(name)
    assert expect in failed, f"{modname}/{mid}: {expect} passes the planted mistake (pins that failed: {failed})"


def test_the_python_pins_pass_on_reloaded_unchanged_modules(monkeypatch):
    """The harness itself: each module re-executed unchanged the same way
    passes its pins."""
    import sys
    import oracle as pkg
    for modname, pins in (("adjoint", ADJ_PINS), ("ssim", SSIM_PINS), ("regularizers", REG_PINS), ("mlp", MLP_PINS),
                          ("densify", DENS_PINS), ("adam", ADAM_PINS)):
        mod = _mutant_module(modname, "", "")
        monkeypatch.setitem(sys.modules, f"oracle.{modname}", mod)
        monkeypatch.setattr(pkg, modname, mod, raising=False)
        if modname == "adjoint":
            monkeypatch.setattr(PINS, "AJ", mod)
        for name in pins:
            _run_pin(name)
