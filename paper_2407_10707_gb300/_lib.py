"""ctypes mirror of include/avatar.h and the loader of libavatar.so.

Argument marshalling only.  The library must exist and a GB300 must be
present; there is no fallback of any kind: every entry point raises if the
native library or the device is missing.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libavatar.so")

P = C.c_void_p
I32 = C.c_int
F32 = C.c_float

STATUS = {0: "AVATAR_OK", 1: "AVATAR_ERR_INVALID_ARG", 2: "AVATAR_ERR_WORKSPACE", 3: "AVATAR_ERR_OVERFLOW",
          4: "AVATAR_ERR_TIMEOUT", 5: "AVATAR_ERR_CUDA", 6: "AVATAR_ERR_UNSUPPORTED", 7: "AVATAR_ERR_INDEX"}


DTYPE_F32 = 0   # avatar_dtype
DTYPE_BF16 = 1
TUNE_BLEND_PPT = 0
TUNE_BLEND_BWD_PPT = 1
TUNE_BATCH_TILE = 2
TUNE_VIS_CLUSTER = 3
TUNE_WAIT_LIMIT = 4
TUNE_REGION_MASKS = 5
VIS_FACE_CHUNK = 1024   # faces per raster chunk (AVATAR_VIS_FACE_CHUNK)
PROBE_FFMA, PROBE_IADD3, PROBE_LOP3, PROBE_IMAD = 0, 1, 2, 3   # avatar_probe_kind


class AvatarError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class SkinArgs(C.Structure):
    _fields_ = [("G", I32), ("Nv", I32), ("K", I32), ("J", I32),
                ("xg", P), ("logscale", P), ("quat", P), ("knn", P),
                ("xv", P), ("dxv", P), ("wv", P), ("av", P), ("rv", P), ("pv", P), ("nv", P),
                ("parents", P), ("joints", P), ("pose", P),
                ("bone", P), ("xp", P), ("xd", P), ("cov", P), ("nd", P), ("ag", P), ("rg", P),
                ("pg", P), ("ubar", P), ("status", P), ("attr_dtype", I32)]


class SkinGrads(C.Structure):
    _fields_ = [("d_xd", P), ("d_cov", P), ("d_nd", P), ("d_ag", P), ("d_rg", P), ("d_pg", P),
                ("d_ubar", P), ("d_xd2", P), ("d_xg", P), ("d_logscale", P), ("d_quat", P), ("d_wv", P),
                ("d_av", P), ("d_rv", P), ("d_pv", P), ("d_dxv", P)]


class VisArgs(C.Structure):
    _fields_ = [("Nv", I32), ("F", I32), ("D", I32), ("R", I32),
                ("xp", P), ("faces", P), ("frames", P),
                ("center", F32 * 3), ("half_extent", F32), ("bias", F32),
                ("NL", I32), ("dmap", P), ("bits", P), ("status", P), ("cull_back", I32)]


class RegArgs(C.Structure):
    _fields_ = [("G", I32), ("Nv", I32), ("Kg", I32), ("Kv", I32), ("xg", P), ("logscale", P), ("knn", P),
                ("xv", P), ("av", P), ("rv", P), ("pv", P), ("knn_v", P), ("dxv", P), ("attr_dtype", I32),
                ("w_smooth", F32), ("w_mdist", F32), ("w_disp", F32), ("w_scale", F32), ("s0", F32),
                ("accumulate", I32), ("loss", P), ("terms", P), ("d_xg", P), ("d_logscale", P), ("d_av", P),
                ("d_rv", P), ("d_pv", P), ("d_dxv", P), ("status", P)]


class MlpArgs(C.Structure):
    _fields_ = [("N", I32), ("P", I32), ("T", I32), ("x", P), ("theta", P), ("Bf", P), ("W1", P), ("b1", P), ("W2", P),
                ("b2", P), ("W3", P), ("b3", P), ("W4", P), ("b4", P), ("dx", P), ("status", P)]


class DensifyArgs(C.Structure):
    _fields_ = [("G", I32), ("Nv", I32), ("F", I32), ("Kg", I32), ("knn", P), ("faces", P), ("xv", P),
                ("d0", F32), ("p0", C.c_double), ("capacity", I32), ("rand", P), ("count", P), ("tri", P), ("x", P),
                ("Dv", P), ("df", P), ("ng", P), ("status", P)]


ADAM_MAX_GROUPS = 16


class AdamGroup(C.Structure):
    _fields_ = [("n", C.c_int64), ("param", P), ("dtype", I32), ("grad", P), ("m", P), ("v", P), ("lr", F32)]


class AdamArgs(C.Structure):
    _fields_ = [("n_groups", I32), ("group", AdamGroup * ADAM_MAX_GROUPS), ("beta1", F32), ("beta2", F32),
                ("eps", F32), ("step", I32)]


class ImageLossArgs(C.Structure):
    _fields_ = [("C", I32), ("H", I32), ("W", I32), ("img", P), ("target", P), ("lam", F32), ("weight", F32),
                ("accumulate", I32), ("loss", P), ("d_img", P)]


class KnnArgs(C.Structure):
    _fields_ = [("N", I32), ("M", I32), ("K", I32), ("x", P), ("ref", P), ("knn", P), ("dist2", P), ("status", P)]


class VisSoftArgs(C.Structure):
    _fields_ = [("base", VisArgs), ("Kv", I32), ("knn_v", P), ("vis_count", P)]


class ShadeArgs(C.Structure):
    _fields_ = [("G", I32), ("K", I32), ("NL", I32), ("Nv", I32),
                ("xd", P), ("nd", P), ("ag", P), ("rg", P), ("pg", P), ("ubar", P), ("knn", P),
                ("bits", P), ("light_L", P), ("light_A", P), ("light_w", P),
                ("cam_center", F32 * 3), ("color", P), ("radiance", P), ("cull", P), ("status", P),
                ("vis_count", P), ("vis_den", I32)]


class ShadeMultiArgs(C.Structure):
    _fields_ = [("base", ShadeArgs), ("n_env", I32), ("env_L", P), ("env_color", P), ("workspace", P),
                ("workspace_bytes", C.c_size_t)]


class ShadeGrads(C.Structure):
    _fields_ = [("d_color", P), ("d_xd", P), ("d_nd", P), ("d_ag", P), ("d_rg", P), ("d_pg", P),
                ("d_ubar", P), ("d_light_L", P)]


class Camera(C.Structure):
    _fields_ = [("fx", F32), ("fy", F32), ("cx", F32), ("cy", F32), ("R", F32 * 9), ("t", F32 * 3),
                ("width", I32), ("height", I32)]


class SplatArgs(C.Structure):
    _fields_ = [("G", I32), ("cam", Camera), ("tile", I32),
                ("xd", P), ("cov", P), ("opacity", P), ("color", P), ("cull", P),
                ("mean2d", P), ("conic", P), ("depth", P), ("rect", P),
                ("tile_range", P), ("pair_gauss", P), ("pair_capacity", C.c_int64), ("num_pairs", P),
                ("image", P), ("T_final", P), ("n_last", P), ("status", P), ("attr_dtype", I32)]


class View(C.Structure):
    _fields_ = [("cam", Camera), ("pose", I32), ("center", F32 * 3)]


class BatchDesc(C.Structure):
    _fields_ = [("avatar", SkinArgs), ("opacity", P),
                ("F", I32), ("faces", P), ("D", I32), ("R", I32), ("frames", P), ("center", F32 * 3),
                ("half_extent", F32), ("bias", F32), ("cull_back", I32),
                ("NL", I32), ("light_A", P), ("light_w", P), ("dmap", P),
                ("B", I32), ("poses", P), ("light_L", P), ("V", I32), ("views", P), ("tile", I32),
                ("pair_capacity", C.c_int64), ("images", P), ("num_pairs", P), ("status", P)]


class BatchGrads(C.Structure):
    _fields_ = [("d_images", P), ("d_xg", P), ("d_logscale", P), ("d_quat", P), ("d_opacity", P), ("d_wv", P),
                ("d_av", P), ("d_rv", P), ("d_pv", P), ("d_light_L", P)]


class SplatGrads(C.Structure):
    _fields_ = [("d_image", P), ("d_xd", P), ("d_cov", P), ("d_opacity", P), ("d_color", P)]


# (name, argtypes, restype)
_SIGNATURES = [
    ("avatar_status_string", [I32], C.c_char_p),
    ("avatar_version", [], I32),
    ("avatar_ctx_create", [C.POINTER(P), I32], I32),
    ("avatar_ctx_destroy", [P], I32),
    ("avatar_ctx_sm_count", [P], I32),
    ("avatar_ctx_set_tuning", [P, I32, I32], I32),
    ("avatar_ctx_get_tuning", [P, I32], I32),
    ("avatar_skin_workspace_size", [C.POINTER(SkinArgs)], C.c_size_t),
    ("avatar_skin", [P, C.POINTER(SkinArgs), P, C.c_size_t, P], I32),
    ("avatar_skin_backward_workspace_size", [C.POINTER(SkinArgs)], C.c_size_t),
    ("avatar_skin_backward", [P, C.POINTER(SkinArgs), C.POINTER(SkinGrads), P, P, C.c_size_t, P], I32),
    ("avatar_visibility_workspace_size", [C.POINTER(VisArgs)], C.c_size_t),
    ("avatar_visibility", [P, C.POINTER(VisArgs), P, C.c_size_t, P], I32),
    ("avatar_visibility_static_scratch_bytes", [], C.c_size_t),
    ("avatar_visibility_static_scratch", [P, C.POINTER(VisArgs), P], I32),
    ("avatar_shade", [P, C.POINTER(ShadeArgs), P], I32),
    ("avatar_cull", [P, C.POINTER(ShadeArgs), P], I32),
    ("avatar_shade_backward", [P, C.POINTER(ShadeArgs), C.POINTER(ShadeGrads), P], I32),
    ("avatar_knn_workspace_size", [C.POINTER(KnnArgs)], C.c_size_t),
    ("avatar_knn", [P, C.POINTER(KnnArgs), P, C.c_size_t, P], I32),
    ("avatar_visibility_soft_workspace_size", [C.POINTER(VisSoftArgs)], C.c_size_t),
    ("avatar_visibility_soft", [P, C.POINTER(VisSoftArgs), P, C.c_size_t, P], I32),
    ("avatar_shade_multi_workspace_size", [C.POINTER(ShadeMultiArgs)], C.c_size_t),
    ("avatar_shade_multi", [P, C.POINTER(ShadeMultiArgs), P], I32),
    ("avatar_splat_num_tiles", [C.POINTER(SplatArgs)], I32),
    ("avatar_splat_workspace_size", [C.POINTER(SplatArgs)], C.c_size_t),
    ("avatar_splat_project", [P, C.POINTER(SplatArgs), P, C.c_size_t, P], I32),
    ("avatar_splat_bin", [P, C.POINTER(SplatArgs), P, C.c_size_t, P], I32),
    ("avatar_splat_blend", [P, C.POINTER(SplatArgs), P, C.c_size_t, P], I32),
    ("avatar_splat", [P, C.POINTER(SplatArgs), P, C.c_size_t, P], I32),
    ("avatar_splat_backward", [P, C.POINTER(SplatArgs), C.POINTER(SplatGrads), P, C.c_size_t, P], I32),
    ("avatar_render_batch_workspace_size", [C.POINTER(BatchDesc)], C.c_size_t),
    ("avatar_render_batch", [P, C.POINTER(BatchDesc), P, C.c_size_t, P], I32),
    ("avatar_render_batch_backward", [P, C.POINTER(BatchDesc), C.POINTER(BatchGrads), P, C.c_size_t, P], I32),
    ("avatar_render_batch_autotune", [P, C.POINTER(BatchDesc), C.POINTER(BatchGrads), P, C.c_size_t, P,
                                      C.POINTER(C.c_int)], I32),
    ("avatar_l1_loss", [P, C.c_int64, P, P, P, P, P], I32),
    ("avatar_regularizers_workspace_size", [C.POINTER(RegArgs)], C.c_size_t),
    ("avatar_regularizers", [P, C.POINTER(RegArgs), P, C.c_size_t, P], I32),
    ("avatar_mlp_workspace_size", [C.POINTER(MlpArgs)], C.c_size_t),
    ("avatar_mlp", [P, C.POINTER(MlpArgs), P, C.c_size_t, P], I32),
    ("avatar_densify_workspace_size", [C.POINTER(DensifyArgs)], C.c_size_t),
    ("avatar_densify", [P, C.POINTER(DensifyArgs), P, C.c_size_t, P], I32),
    ("avatar_adam", [P, C.POINTER(AdamArgs), P], I32),
    ("avatar_image_loss_workspace_size", [C.POINTER(ImageLossArgs)], C.c_size_t),
    ("avatar_image_loss", [P, C.POINTER(ImageLossArgs), P, C.c_size_t, P], I32),
    ("avatar_probe_alu", [P, I32, I32, P, C.POINTER(C.c_longlong), P], I32),
    ("avatar_gaussian_order_workspace_size", [I32], C.c_size_t),
    ("avatar_gaussian_order", [P, I32, I32, P, P, P, C.c_size_t, P, P], I32),
    ("avatar_gather_columns", [P, I32, I32, I32, P, P, P, P, P], I32),
]

EXPORTED = [s[0] for s in _SIGNATURES]

_lib = None


def load(path: str = LIB_PATH):
    """Load libavatar.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                           "(the CUDA library is required; there is no CPU path)")
    lib = C.CDLL(path)
    for name, args, res in _SIGNATURES:
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(rc: int, where: str):
    if rc != 0:
        raise AvatarError(rc, where)
