"""ctypes front end of the FP64 C oracle (avatar_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  Inputs are taken as
numpy arrays in the oracle's own AoS layout and converted to float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "avatar_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _lib.orc_bin.restype = ctypes.c_long
        _lib.orc_visibility.restype = ctypes.c_int
        _lib.orc_visibility_tri.restype = ctypes.c_int
        _lib.orc_vis_filter.restype = ctypes.c_int
        _lib.orc_knn.restype = ctypes.c_int
        _lib.orc_set_threads.restype = ctypes.c_int
    return _lib


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def fk(parents, joints, pose):
    J = len(parents)
    bone = np.zeros((J, 3, 4))
    parents, joints, pose = _i(parents), _d(joints), _d(pose)
    lib().orc_fk(ctypes.c_int(J), _p(parents), _p(joints), _p(pose), _p(bone))
    return bone


def skin(av, bone):
    """av: synth.Avatar; bone: [J,3,4].  Returns dict of FP64 outputs."""
    G, Nv, K, J = av.G, av.Nv, av.K, bone.shape[0]
    ins = dict(xg=_d(av.xg), ls=_d(av.logscale), q=_d(av.quat), knn=_i(av.knn), xv=_d(av.xv),
               dxv=_d(av.dxv), wv=_d(av.wv), a=_d(av.av), r=_d(av.rv), p=_d(av.pv), n=_d(av.nv),
               bone=_d(bone))
    out = dict(xp=np.zeros((Nv, 3)), xd=np.zeros((G, 3)), cov=np.zeros((G, 6)),
               nd=np.zeros((G, 3)), ag=np.zeros((G, 3)), rg=np.zeros(G), pg=np.zeros(G),
               ubar=np.zeros((G, K)), wg=np.zeros((G, J)))
    lib().orc_skin(ctypes.c_int(G), ctypes.c_int(Nv), ctypes.c_int(K), ctypes.c_int(J),
                   _p(ins["xg"]), _p(ins["ls"]), _p(ins["q"]), _p(ins["knn"]), _p(ins["xv"]),
                   _p(ins["dxv"]), _p(ins["wv"]), _p(ins["a"]), _p(ins["r"]), _p(ins["p"]),
                   _p(ins["n"]), _p(ins["bone"]), _p(out["xp"]), _p(out["xd"]), _p(out["cov"]),
                   _p(out["nd"]), _p(out["ag"]), _p(out["rg"]), _p(out["pg"]), _p(out["ubar"]),
                   _p(out["wg"]))
    return out


def visibility(xp, faces, frames, center, half_extent, bias, depth_res, want_depth=False, cull_back=False):
    """Exact integer visibility bits [Nv, D/32] (uint32); raises on bad args."""
    xp, faces, frames = _d(xp), _i(faces), _d(np.asarray(frames).reshape(-1, 9))
    center = _d(center)
    Nv, F, D = xp.shape[0], faces.shape[0], frames.shape[0]
    bits = np.zeros((Nv, D // 32), dtype=np.uint32)
    depth = np.zeros((D, depth_res, depth_res), dtype=np.int32) if want_depth else None
    rc = lib().orc_visibility(ctypes.c_int(Nv), ctypes.c_int(F), ctypes.c_int(D),
                              ctypes.c_int(depth_res), _p(xp), _p(faces), _p(frames), _p(center),
                              ctypes.c_double(half_extent), ctypes.c_double(bias),
                              ctypes.c_int(1 if cull_back else 0), _p(bits), _p(depth))
    if rc != 0:
        raise ValueError("oracle visibility: argument outside the supported range")
    return (bits, depth) if want_depth else bits


def knn(x, ref, k, want_dist=False):
    """Indices [N, k] of the k nearest reference points of every query point,
    ascending (squared distance, index); x, ref are rounded to FP32 first
    (the values an FP32 stage holds), distances exact in FP64."""
    x = _d(np.asarray(x, np.float32))
    ref = _d(np.asarray(ref, np.float32))
    N, M = x.shape[0], ref.shape[0]
    out = np.zeros((N, k), np.int32)
    d2 = np.zeros((N, k)) if want_dist else None
    rc = lib().orc_knn(ctypes.c_int(N), ctypes.c_int(M), ctypes.c_int(k), _p(x), _p(ref), _p(out), _p(d2))
    if rc != 0:
        raise ValueError("oracle knn: bad sizes")
    return (out, d2) if want_dist else out


def visibility_tri(xp, faces, frames, center, half_extent, depth_res, cull_back=False, want_tri=False):
    """The paper's triangle-ID visibility V [Nv, D/32] (uint32 bits), Sec. 3.2."""
    xp, faces, frames = _d(xp), _i(faces), _d(np.asarray(frames).reshape(-1, 9))
    center = _d(center)
    Nv, F, D = xp.shape[0], faces.shape[0], frames.shape[0]
    bits = np.zeros((Nv, D // 32), dtype=np.uint32)
    tri = np.zeros((D, depth_res, depth_res), dtype=np.int32) if want_tri else None
    rc = lib().orc_visibility_tri(ctypes.c_int(Nv), ctypes.c_int(F), ctypes.c_int(D), ctypes.c_int(depth_res),
                                  _p(xp), _p(faces), _p(frames), _p(center), ctypes.c_double(half_extent),
                                  ctypes.c_int(1 if cull_back else 0), _p(bits), _p(tri))
    if rc != 0:
        raise ValueError("oracle triangle-ID visibility: argument outside the supported range")
    return (bits, tri) if want_tri else bits


def vis_filter(bits, knn_v):
    """Kv * mean(median(median(V))) per vertex and direction (Eqs. 3-4), uint8 [Nv, D].
    knn_v: [Nv, Kv] nearest vertices of each vertex (itself included)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    knn_v = _i(knn_v)
    Nv, DW = bits.shape
    Kv = knn_v.shape[1]
    out = np.zeros((Nv, DW * 32), np.uint8)
    rc = lib().orc_vis_filter(ctypes.c_int(Nv), ctypes.c_int(DW * 32), ctypes.c_int(Kv), _p(knn_v), _p(bits),
                              _p(out))
    if rc != 0:
        raise ValueError("oracle visibility filter: bad sizes or indices")
    return out


def brdf_terms(gamma, nh, voh, ci, co, library=None):
    """App. A terms (D, F, G, f_s) of the specular BRDF at roughness gamma for
    the cosines n.h, w_o.h, n.w_i, n.w_o; f_s is the value the shading sums.
    library: another build of the oracle source (a ctypes CDLL), else this one."""
    L = library if library is not None else lib()
    out = np.zeros(4)
    L.orc_brdf_terms(ctypes.c_double(gamma), ctypes.c_double(nh), ctypes.c_double(voh), ctypes.c_double(ci),
                     ctypes.c_double(co), _p(out))
    return out


def shade_soft(xd, nd, ag, rg, pg, ubar, knn, vis_count, vis_den, light_L, light_A, light_w, dmap, cam_center):
    """Shading with soft vertex visibility vis_count [Nv, D] / vis_den."""
    xd, nd, ag, rg, pg, ubar = map(_d, (xd, nd, ag, rg, pg, ubar))
    knn, dmap = _i(knn), _i(dmap)
    vc = np.ascontiguousarray(vis_count, dtype=np.uint8)
    light_L, light_A, light_w, cam_center = map(_d, (light_L, light_A, light_w, cam_center))
    G, K, NL = xd.shape[0], knn.shape[1], light_L.shape[0]
    color = np.zeros((G, 3))
    radiance = np.zeros((G, 3))
    cull = np.zeros(G, dtype=np.uint8)
    lib().orc_shade_soft(ctypes.c_int(G), ctypes.c_int(K), ctypes.c_int(NL), ctypes.c_int(vc.shape[1]),
                         _p(xd), _p(nd), _p(ag), _p(rg), _p(pg), _p(ubar), _p(knn), _p(vc), ctypes.c_int(vis_den),
                         _p(light_L), _p(light_A), _p(light_w), _p(dmap), _p(cam_center), _p(color), _p(radiance),
                         _p(cull))
    return color, radiance, cull


def shade(xd, nd, ag, rg, pg, ubar, knn, bits, light_L, light_A, light_w, dmap, cam_center,
          n_dirs):
    xd, nd, ag, rg, pg, ubar = map(_d, (xd, nd, ag, rg, pg, ubar))
    knn, dmap = _i(knn), _i(dmap)
    bits = np.ascontiguousarray(bits, dtype=np.uint32)
    light_L, light_A, light_w, cam_center = map(_d, (light_L, light_A, light_w, cam_center))
    G, K, NL = xd.shape[0], knn.shape[1], light_L.shape[0]
    color = np.zeros((G, 3))
    radiance = np.zeros((G, 3))
    cull = np.zeros(G, dtype=np.uint8)
    lib().orc_shade(ctypes.c_int(G), ctypes.c_int(K), ctypes.c_int(NL), ctypes.c_int(n_dirs),
                    _p(xd), _p(nd), _p(ag), _p(rg), _p(pg), _p(ubar), _p(knn), _p(bits),
                    _p(light_L), _p(light_A), _p(light_w), _p(dmap), _p(cam_center),
                    _p(color), _p(radiance), _p(cull))
    return color, radiance, cull


def camera_vector(cam):
    return _d(np.concatenate([[cam.fx, cam.fy, cam.cx, cam.cy], np.asarray(cam.R).reshape(-1),
                              np.asarray(cam.t).reshape(-1)]))


def project(xd, cov, opacity, cull, cam):
    xd, cov, opacity = _d(xd), _d(cov), _d(opacity)
    G = xd.shape[0]
    cull = np.zeros(G, np.uint8) if cull is None else np.ascontiguousarray(cull, np.uint8)
    camv = camera_vector(cam)
    out = dict(mean2d=np.zeros((G, 2)), conic=np.zeros((G, 3)), depth=np.zeros(G),
               rect=np.zeros((G, 4), np.int32), valid=np.zeros(G, np.int32),
               rect_amb=np.zeros(G, np.uint8))
    lib().orc_project(ctypes.c_int(G), _p(xd), _p(cov), _p(opacity), _p(cull), _p(camv),
                      ctypes.c_int(cam.width), ctypes.c_int(cam.height), _p(out["mean2d"]),
                      _p(out["conic"]), _p(out["depth"]), _p(out["rect"]), _p(out["valid"]),
                      _p(out["rect_amb"]))
    return out


def composite(mean2d, conic, opacity, color, depth, valid, width, height, pixels=None):
    """Brute-force compositing; pixels = optional array of flat pixel indices."""
    mean2d, conic, opacity, color, depth = map(_d, (mean2d, conic, opacity, color, depth))
    valid = _i(valid)
    G = mean2d.shape[0]
    if pixels is None:
        n, pix = width * height, None
    else:
        pix = _i(pixels)
        n = len(pix)
    rgb = np.zeros((n, 3))
    T = np.zeros(n)
    count = np.zeros(n, np.int32)
    amb = np.zeros(n, np.uint8)
    lib().orc_composite(ctypes.c_int(G), ctypes.c_int(width), ctypes.c_int(height), _p(mean2d),
                        _p(conic), _p(opacity), _p(color), _p(depth), _p(valid), ctypes.c_int(n),
                        _p(pix), _p(rgb), _p(T), _p(count), _p(amb))
    return rgb, T, count, amb


def bin_tiles(rect, depth_key, width, height, tile):
    rect = _i(rect)
    key = np.ascontiguousarray(depth_key, dtype=np.uint32)
    G = rect.shape[0]
    ntiles = ((width + tile - 1) // tile) * ((height + tile - 1) // tile)
    start = np.zeros(ntiles + 1, np.int32)
    cap = 1 << 16
    while True:
        lst = np.zeros(cap, np.int32)
        total = lib().orc_bin(ctypes.c_int(G), _p(rect), _p(key), ctypes.c_int(width),
                              ctypes.c_int(height), ctypes.c_int(tile), _p(start), _p(lst),
                              ctypes.c_long(cap))
        if total <= cap:
            return start, lst[:total]
        cap = int(total)
