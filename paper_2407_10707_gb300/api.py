"""PyTorch-facing binding of the C ABI (include/avatar.h), same names.

Each function marshals torch CUDA tensors (float32 structure-of-arrays,
int32 indices) into the argument structs and calls the native entry point
on the current stream.  Outputs that are not passed in are allocated with
torch (the library itself never allocates).  No arithmetic of the render
path happens here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need_cuda(t, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


_CTX = {}


def context(device=None):
    """The avatar_ctx of a CUDA device (created once per device)."""
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device (GB300, sm_103a) is required: the render path has no CPU fallback")
    lib = L.load()
    dev = torch.cuda.current_device() if device is None else torch.device(device).index or 0
    if dev not in _CTX:
        h = C.c_void_p()
        L.check(lib.avatar_ctx_create(C.byref(h), dev), "avatar_ctx_create")
        _CTX[dev] = h
    return _CTX[dev]


def workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def status_word(device):
    return torch.zeros(1, dtype=torch.int32, device=device)


def raise_on_status(status, where="device"):
    v = int(status.item())
    if v != 0:
        raise L.AvatarError(v, where)


# ---------------------------------------------------------------- inputs
# Learnable attributes that may be stored in BF16 (AVATAR_DTYPE_BF16).
ATTR_KEYS = ("logscale", "quat", "opacity", "av", "rv", "pv")


def avatar_tensors(av, device="cuda", attr_dtype="f32"):
    """Device layout of a synth.Avatar: SoA float32, int32 indices; with
    attr_dtype='bf16' the ATTR_KEYS tensors are stored as bfloat16."""
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    i = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.int32, device=device)
    t = dict(xg=f(av.xg.T), logscale=f(av.logscale.T), quat=f(av.quat.T), opacity=f(av.opacity),
             knn=i(av.knn.T), xv=f(av.xv.T), dxv=f(av.dxv.T), wv=f(av.wv), av=f(av.av.T), rv=f(av.rv),
             pv=f(av.pv), nv=f(av.nv.T), parents=i(av.parents), joints=f(av.joints), pose=f(av.pose),
             faces=i(av.faces))
    if attr_dtype == "bf16":
        for k in ATTR_KEYS:
            t[k] = t[k].to(torch.bfloat16)
    elif attr_dtype != "f32":
        raise ValueError(f"attr_dtype must be 'f32' or 'bf16', not {attr_dtype!r}")
    return t


def _dtype_code(*tensors):
    """AVATAR_DTYPE_* of the attribute tensors given (all must agree)."""
    kinds = {x.dtype for x in tensors if x is not None}
    if not kinds:
        return L.DTYPE_F32
    if len(kinds) > 1 or not kinds <= {torch.float32, torch.bfloat16}:
        raise ValueError(f"attribute tensors must all be float32 or all bfloat16, got {sorted(map(str, kinds))}")
    return L.DTYPE_BF16 if kinds == {torch.bfloat16} else L.DTYPE_F32


def camera_struct(cam):
    c = L.Camera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float32).reshape(-1)
    t = np.asarray(cam.t, np.float32).reshape(-1)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.width, c.height = int(cam.width), int(cam.height)
    return c


# ---------------------------------------------------------------- (a) skinning
def _skin_struct(t, out, status):
    G = t["xg"].shape[1]
    Nv = t["xv"].shape[1]
    K = t["knn"].shape[0]
    J = t["parents"].shape[0]
    a = L.SkinArgs()
    a.G, a.Nv, a.K, a.J = G, Nv, K, J
    for k in ("xg", "logscale", "quat", "knn", "xv", "dxv", "wv", "av", "rv", "pv", "nv", "parents", "joints",
              "pose"):
        setattr(a, k, _p(t.get(k)))
    for k in ("bone", "xp", "xd", "cov", "nd", "ag", "rg", "pg", "ubar"):
        setattr(a, k, _p(out[k]))
    a.status = _p(status)
    a.attr_dtype = _dtype_code(*(t.get(k) for k in ("logscale", "quat", "av", "rv", "pv")))
    return a


def alloc_skin_outputs(t):
    dev = t["xg"].device
    G, Nv, K, J = t["xg"].shape[1], t["xv"].shape[1], t["knn"].shape[0], t["parents"].shape[0]
    e = lambda *s: torch.empty(*s, dtype=torch.float32, device=dev)
    return dict(bone=e(J, 12), xp=e(3, Nv), xd=e(3, G), cov=e(6, G), nd=e(3, G), ag=e(3, G), rg=e(G), pg=e(G),
                ubar=e(K, G))


def avatar_skin(t, out=None, ws=None, status=None):
    """(a) Skinning (Sec. 3.1, Eq. 1).  Returns the output dict; out['_ws']
    holds the workspace the backward needs."""
    lib = L.load()
    ctx = context()
    out = alloc_skin_outputs(t) if out is None else out
    a = _skin_struct(t, out, status)
    need = lib.avatar_skin_workspace_size(C.byref(a))
    if ws is None or ws.numel() < need:
        ws = workspace(need, t["xg"].device)
    L.check(lib.avatar_skin(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_skin")
    out["_ws"] = ws
    return out


def avatar_skin_backward(t, out, up, want=("xg", "logscale", "quat", "wv", "av", "rv", "pv")):
    """Adjoint of avatar_skin.  up: dict of upstream grads (d_xd, d_xd2,
    d_cov, d_nd, d_ag, d_rg, d_pg, d_ubar; missing = zero)."""
    lib = L.load()
    ctx = context()
    a = _skin_struct(t, out, None)
    dev = t["xg"].device
    g = L.SkinGrads()
    keep = []
    for k in ("d_xd", "d_cov", "d_nd", "d_ag", "d_rg", "d_pg", "d_ubar", "d_xd2"):
        v = up.get(k)
        v = v.contiguous() if v is not None else None
        keep.append(v)
        setattr(g, k, _p(v))
    res = {}
    for k in want:   # gradients are FP32 whatever the storage type
        res[k] = torch.empty_like(t[k], dtype=torch.float32)
        setattr(g, "d_" + k, _p(res[k]))
    need = lib.avatar_skin_backward_workspace_size(C.byref(a))
    ws = workspace(need, dev)
    L.check(lib.avatar_skin_backward(ctx, C.byref(a), C.byref(g), _p(out["_ws"]), _p(ws), ws.numel(), _stream()),
            "avatar_skin_backward")
    del keep
    return res


# ---------------------------------------------------------------- (b) visibility
def _vis_struct(xp, faces, frames, center, half_extent, bias, R, dmap, bits, status, cull_back=False):
    a = L.VisArgs()
    a.Nv = xp.shape[1]
    a.F = faces.shape[0]
    a.D = frames.shape[0]
    a.R = int(R)
    a.xp, a.faces, a.frames = _p(xp), _p(faces), _p(frames)
    for k in range(3):
        a.center[k] = float(center[k])
    a.half_extent = float(half_extent)
    a.bias = float(bias)
    a.NL = 0 if dmap is None else dmap.shape[0]
    a.dmap = _p(dmap)
    a.bits = _p(bits)
    a.status = _p(status)
    a.cull_back = 1 if cull_back else 0
    return a


def avatar_visibility(xp, faces, frames, center, half_extent, bias, R, dmap=None, bits=None, ws=None,
                      status=None, cull_back=False):
    """(b) Depth-map visibility bits (Sec. 3.2).  xp [3,Nv] f32, faces [F,3]
    i32, frames [D,9] f32.  Returns uint32-valued int32 words, light-ordered
    [Nv, ceil(NL/32)] when dmap is given, else [Nv, D/32]."""
    lib = L.load()
    ctx = context()
    Nv = xp.shape[1]
    nout = dmap.shape[0] if dmap is not None else frames.shape[0]
    if bits is None:
        bits = torch.empty(Nv, (nout + 31) // 32, dtype=torch.int32, device=xp.device)
    a = _vis_struct(xp, faces, frames, center, half_extent, bias, R, dmap, bits, status, cull_back)
    need = lib.avatar_visibility_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_visibility_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, xp.device)
    L.check(lib.avatar_visibility(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_visibility")
    return bits


def avatar_knn(x, ref, k, out=None, dist2=None, ws=None, status=None):
    """Indices [k, N] of the k nearest reference points ([3, M]) of each
    query point ([3, N]), ascending (FP64 squared distance, index)."""
    lib = L.load()
    ctx = context()
    a = L.KnnArgs()
    a.N, a.M, a.K = x.shape[1], ref.shape[1], int(k)
    if out is None:
        out = torch.empty(k, a.N, dtype=torch.int32, device=x.device)
    a.x, a.ref, a.knn, a.dist2, a.status = _p(x), _p(ref), _p(out), _p(dist2), _p(status)
    need = lib.avatar_knn_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_knn_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    L.check(lib.avatar_knn(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_knn")
    return out


def avatar_visibility_soft(xp, faces, frames, center, half_extent, R, knn_v, dmap=None, vis_count=None,
                           raw_bits=None, ws=None, status=None, cull_back=False):
    """(b') The paper's visibility (Sec. 3.2, Eqs. 3-4): triangle-ID images and
    the median/median/mean filters over the Kv nearest vertices.  knn_v
    [Kv, Nv] int32.  Returns uint8 counts Kv * Vbar, [Nv, NL] (light order
    when dmap is given, else [Nv, D]); raw_bits, if given ([Nv, D/32] int32),
    receives the unfiltered V in direction order."""
    lib = L.load()
    ctx = context()
    Nv = xp.shape[1]
    nout = dmap.shape[0] if dmap is not None else frames.shape[0]
    if vis_count is None:
        vis_count = torch.empty(Nv, nout, dtype=torch.uint8, device=xp.device)
    a = L.VisSoftArgs()
    a.base = _vis_struct(xp, faces, frames, center, half_extent, 0.0, R, dmap, raw_bits, status, cull_back)
    a.Kv = knn_v.shape[0]
    a.knn_v = _p(knn_v)
    a.vis_count = _p(vis_count)
    need = lib.avatar_visibility_soft_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_visibility_soft_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, xp.device)
    L.check(lib.avatar_visibility_soft(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_visibility_soft")
    return vis_count


# ---------------------------------------------------------------- (c) shading
def _shade_struct(sk, knn, bits, light, cam_center, color, radiance, cull, status, vis_den=None):
    """bits: visibility words (int32) or, for the soft visibility of the
    paper's filters, uint8 counts [Nv, NL] with vis_den = Kv."""
    a = L.ShadeArgs()
    a.G = sk["xd"].shape[1]
    a.K = knn.shape[0]
    a.NL = light["L"].shape[0]
    a.Nv = bits.shape[0]
    a.xd, a.nd, a.ag, a.rg, a.pg, a.ubar = (_p(sk[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar"))
    if bits.dtype == torch.uint8:
        if vis_den is None:
            raise ValueError("soft visibility counts need vis_den (the filters' Kv)")
        a.knn, a.bits = _p(knn), None
        a.vis_count, a.vis_den = _p(bits), int(vis_den)
    else:
        a.knn, a.bits = _p(knn), _p(bits)
    a.light_L, a.light_A, a.light_w = _p(light["L"]), _p(light["A"]), _p(light["w"])
    for k in range(3):
        a.cam_center[k] = float(cam_center[k])
    a.color, a.radiance, a.cull, a.status = _p(color), _p(radiance), _p(cull), _p(status)
    return a


def avatar_shade(sk, knn, bits, light, cam_center, out=None, status=None, vis_den=None):
    """(c) Shading (Eq. 2, App. A).  light: dict L [NL,3], A [NL], w [NL,3];
    bits: visibility words, or uint8 soft counts with vis_den."""
    lib = L.load()
    ctx = context()
    dev = sk["xd"].device
    G = sk["xd"].shape[1]
    if out is None:
        out = dict(color=torch.empty(3, G, device=dev), radiance=torch.empty(3, G, device=dev),
                   cull=torch.empty(G, dtype=torch.uint8, device=dev))
    a = _shade_struct(sk, knn, bits, light, cam_center, out["color"], out["radiance"], out["cull"], status, vis_den)
    L.check(lib.avatar_shade(ctx, C.byref(a), _stream()), "avatar_shade")
    return out


def avatar_cull(sk, cam_center, cull=None):
    """The back-face flags of avatar_shade alone (the same FP32 rule on the
    skinned xd, nd and the camera centre), [G] uint8, 1 = culled."""
    lib = L.load()
    ctx = context()
    G = sk["xd"].shape[1]
    if cull is None:
        cull = torch.empty(G, dtype=torch.uint8, device=sk["xd"].device)
    a = L.ShadeArgs()
    a.G = G
    a.xd, a.nd = _p(sk["xd"]), _p(sk["nd"])
    for k in range(3):
        a.cam_center[k] = float(cam_center[k])
    a.cull = _p(cull)
    L.check(lib.avatar_cull(ctx, C.byref(a), _stream()), "avatar_cull")
    return cull


def avatar_shade_multi(sk, knn, bits, light, cam_center, env_L, out=None, cull=None, status=None, ws=None,
                       radiance=None):
    """Colours under n_env environment lights sharing light['A'], light['w']
    (tensor-core path).  env_L: [n_env, NL, 3].  Returns [n_env, 3, G];
    with n_env == 1, `radiance` ([3, G]) receives L_o before gamma."""
    lib = L.load()
    ctx = context()
    dev = sk["xd"].device
    G = sk["xd"].shape[1]
    n_env = env_L.shape[0]
    env_L = env_L.contiguous()
    if out is None:
        out = torch.empty(n_env, 3, G, device=dev)
    if cull is None:
        cull = torch.empty(G, dtype=torch.uint8, device=dev)
    m = L.ShadeMultiArgs()
    m.base = _shade_struct(sk, knn, bits, dict(light, L=light.get("L", env_L[0])), cam_center, None, radiance, cull,
                           status)
    m.n_env = n_env
    m.env_L = _p(env_L)
    m.env_color = _p(out)
    need = lib.avatar_shade_multi_workspace_size(C.byref(m))
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    m.workspace, m.workspace_bytes = _p(ws), ws.numel()
    L.check(lib.avatar_shade_multi(ctx, C.byref(m), _stream()), "avatar_shade_multi")
    return out


def avatar_shade_backward(sk, knn, bits, light, cam_center, out, d_color, vis_den=None):
    lib = L.load()
    ctx = context()
    a = _shade_struct(sk, knn, bits, light, cam_center, out["color"], out["radiance"], out["cull"], None, vis_den)
    d_color = d_color.contiguous()
    res = dict(xd=torch.empty_like(sk["xd"]), nd=torch.empty_like(sk["nd"]), ag=torch.empty_like(sk["ag"]),
               rg=torch.empty_like(sk["rg"]), pg=torch.empty_like(sk["pg"]), ubar=torch.empty_like(sk["ubar"]),
               L=torch.empty_like(light["L"]))
    g = L.ShadeGrads()
    g.d_color = _p(d_color)
    g.d_xd, g.d_nd, g.d_ag, g.d_rg, g.d_pg, g.d_ubar, g.d_light_L = (
        _p(res[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar", "L"))
    L.check(lib.avatar_shade_backward(ctx, C.byref(a), C.byref(g), _stream()), "avatar_shade_backward")
    return res


# ---------------------------------------------------------------- (d) splatting
@dataclass
class SplatBuffers:
    mean2d: torch.Tensor
    conic: torch.Tensor
    depth: torch.Tensor
    rect: torch.Tensor
    tile_range: torch.Tensor
    pair_gauss: torch.Tensor
    num_pairs: torch.Tensor
    image: torch.Tensor
    T_final: torch.Tensor
    n_last: torch.Tensor
    ws: torch.Tensor
    tile: int


def num_tiles(width, height, tile):
    return ((width + tile - 1) // tile) * ((height + tile - 1) // tile)


def alloc_splat(G, cam, tile=16, pair_capacity=None, device="cuda"):
    tile = tile or 16
    W, H = int(cam.width), int(cam.height)
    # default pair capacity: 32 tiles per Gaussian at 16-pixel tiles, four
    # times that at 8 (a Gaussian's tile count grows with the inverse square
    # of the tile edge); overflow is reported on the status word, not written
    cap = int(pair_capacity or max(1 << 16, 32 * G * (4 if tile == 8 else 1)))
    e = lambda *s, dt=torch.float32: torch.empty(*s, dtype=dt, device=device)
    b = SplatBuffers(mean2d=e(2, G), conic=e(3, G), depth=e(G), rect=e(4, G, dt=torch.int32),
                     tile_range=e(num_tiles(W, H, tile), 2, dt=torch.int32), pair_gauss=e(cap, dt=torch.int32),
                     num_pairs=e(1, dt=torch.int32), image=e(3, H, W), T_final=e(H, W),
                     n_last=e(H, W, dt=torch.int32), ws=None, tile=tile)
    a = _splat_struct(G, cam, None, None, None, None, None, b, None)
    need = L.load().avatar_splat_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_splat_workspace_size")
    b.ws = workspace(need, device)
    return b


def _splat_struct(G, cam, xd, cov, opacity, color, cull, b: SplatBuffers, status):
    a = L.SplatArgs()
    a.G = G
    a.cam = camera_struct(cam)
    a.tile = b.tile
    a.xd, a.cov, a.opacity, a.color, a.cull = _p(xd), _p(cov), _p(opacity), _p(color), _p(cull)
    a.mean2d, a.conic, a.depth, a.rect = _p(b.mean2d), _p(b.conic), _p(b.depth), _p(b.rect)
    a.tile_range, a.pair_gauss, a.num_pairs = _p(b.tile_range), _p(b.pair_gauss), _p(b.num_pairs)
    a.pair_capacity = b.pair_gauss.numel()
    a.image, a.T_final, a.n_last = _p(b.image), _p(b.T_final), _p(b.n_last)
    a.status = _p(status)
    a.attr_dtype = _dtype_code(opacity)
    return a


def _splat_call(name, xd, cov, opacity, color, cull, cam, b, status):
    lib = L.load()
    ctx = context()
    G = xd.shape[1]
    a = _splat_struct(G, cam, xd, cov, opacity, color, cull, b, status)
    L.check(getattr(lib, name)(ctx, C.byref(a), _p(b.ws), b.ws.numel(), _stream()), name)
    return b


def avatar_splat_project(xd, cov, opacity, color, cull, cam, b, status=None):
    return _splat_call("avatar_splat_project", xd, cov, opacity, color, cull, cam, b, status)


def avatar_splat_bin(xd, cov, opacity, color, cull, cam, b, status=None):
    return _splat_call("avatar_splat_bin", xd, cov, opacity, color, cull, cam, b, status)


def avatar_splat_blend(xd, cov, opacity, color, cull, cam, b, status=None):
    return _splat_call("avatar_splat_blend", xd, cov, opacity, color, cull, cam, b, status)


def avatar_splat(xd, cov, opacity, color, cull, cam, b=None, tile=16, pair_capacity=None, status=None):
    """(d) Splatting (3DGS rasteriser of Sec. 3.1).  Returns SplatBuffers."""
    if b is None:
        b = alloc_splat(xd.shape[1], cam, tile, pair_capacity, xd.device)
    return _splat_call("avatar_splat", xd, cov, opacity, color, cull, cam, b, status)


def avatar_splat_backward(xd, cov, opacity, color, cull, cam, b, d_image):
    lib = L.load()
    ctx = context()
    G = xd.shape[1]
    a = _splat_struct(G, cam, xd, cov, opacity, color, cull, b, None)
    d_image = d_image.contiguous()
    res = dict(xd=torch.empty_like(xd), cov=torch.empty_like(cov),
               opacity=torch.empty_like(opacity, dtype=torch.float32), color=torch.empty_like(color))
    g = L.SplatGrads()
    g.d_image = _p(d_image)
    g.d_xd, g.d_cov, g.d_opacity, g.d_color = _p(res["xd"]), _p(res["cov"]), _p(res["opacity"]), _p(res["color"])
    L.check(lib.avatar_splat_backward(ctx, C.byref(a), C.byref(g), _p(b.ws), b.ws.numel(), _stream()),
            "avatar_splat_backward")
    return res


# ---------------------------------------------------------------- loss
def avatar_l1_loss(img, target, want_grad=True):
    lib = L.load()
    ctx = context()
    img = img.contiguous()
    target = target.contiguous()
    loss = torch.empty(1, dtype=torch.float32, device=img.device)
    d_img = torch.empty_like(img) if want_grad else None
    L.check(lib.avatar_l1_loss(ctx, img.numel(), _p(img), _p(target), _p(loss), _p(d_img), _stream()),
            "avatar_l1_loss")
    return loss, d_img


def avatar_image_loss(img, target, lam=0.2, d_img=None, loss=None, ws=None, weight=1.0, accumulate=False,
                      want_grad=True):
    """Eq. 5's image loss (1 - lam) L1 + lam D-SSIM of img, target [C, H, W].
    Returns (loss [1], d_img)."""
    lib = L.load()
    ctx = context()
    img = img.contiguous()
    target = target.contiguous()
    a = L.ImageLossArgs()
    a.C, a.H, a.W = img.shape
    a.img, a.target = _p(img), _p(target)
    a.lam, a.weight, a.accumulate = float(lam), float(weight), 1 if accumulate else 0
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float32, device=img.device)
    if want_grad and d_img is None:
        d_img = torch.empty_like(img)
    a.loss, a.d_img = _p(loss), _p(d_img) if want_grad else None
    need = lib.avatar_image_loss_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_image_loss_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, img.device)
    L.check(lib.avatar_image_loss(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_image_loss")
    return loss, d_img


REG_WEIGHTS = dict(smooth=0.002, mdist=0.1, disp=0.02, scale=10.0)  # Sec. 3.3


def avatar_regularizers(t, knn_v, grads=None, loss=None, terms=None, weights=None, s0=0.005, accumulate=False,
                        ws=None, status=None):
    """Sec. 3.3's regularisers of the avatar tensors t (avatar_tensors layout)
    with the vertex neighbourhoods knn_v [Kv, Nv].  grads: dict of FP32
    buffers (xg, logscale, av, rv, pv, dxv) the gradients are ADDED to.
    Returns (loss [1], terms [4])."""
    lib = L.load()
    ctx = context()
    w = dict(REG_WEIGHTS if weights is None else weights)
    dev = t["xg"].device
    a = L.RegArgs()
    a.G, a.Nv = t["xg"].shape[1], t["xv"].shape[1]
    a.Kg, a.Kv = t["knn"].shape[0], knn_v.shape[0]
    a.xg, a.logscale, a.knn, a.xv = _p(t["xg"]), _p(t["logscale"]), _p(t["knn"]), _p(t["xv"])
    a.av, a.rv, a.pv, a.knn_v, a.dxv = _p(t["av"]), _p(t["rv"]), _p(t["pv"]), _p(knn_v), _p(t.get("dxv"))
    a.attr_dtype = _dtype_code(t["logscale"], t["av"], t["rv"], t["pv"])
    a.w_smooth, a.w_mdist, a.w_disp, a.w_scale, a.s0 = w["smooth"], w["mdist"], w["disp"], w["scale"], float(s0)
    a.accumulate = 1 if accumulate else 0
    if loss is None:
        loss = torch.zeros(1, device=dev)
    if terms is None:
        terms = torch.zeros(4, device=dev)
    a.loss, a.terms, a.status = _p(loss), _p(terms), _p(status)
    grads = grads or {}
    a.d_xg, a.d_logscale, a.d_av = _p(grads.get("xg")), _p(grads.get("logscale")), _p(grads.get("av"))
    a.d_rv, a.d_pv, a.d_dxv = _p(grads.get("rv")), _p(grads.get("pv")), _p(grads.get("dxv"))
    need = lib.avatar_regularizers_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_regularizers_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    L.check(lib.avatar_regularizers(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_regularizers")
    return loss, terms


# ---------------------------------------------------------------- displacement MLP
MLP_KEYS = ("Bf", "W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def mlp_tensors(w, device):
    """The MLP's weights (dict of arrays, MLP_KEYS) as contiguous FP32 device tensors."""
    return {k: torch.as_tensor(np.asarray(w[k]), dtype=torch.float32).contiguous().to(device) for k in MLP_KEYS}


def mlp_workspace_size(n, p, t=1):
    a = L.MlpArgs()
    a.N, a.P, a.T = n, p, t
    return L.load().avatar_mlp_workspace_size(C.byref(a))


def avatar_mlp(x, theta, w, dx=None, ws=None, status=None):
    """Sec. 3.1's displacement dx [3, N] of the points x [3, N] at pose
    theta [P], or its mean over the poses theta [T, P] (Sec. 4's average
    displacement); weights w from mlp_tensors."""
    lib = L.load()
    ctx = context()
    x = x.contiguous()
    theta = theta.contiguous()
    if theta.dim() == 1:
        theta = theta.unsqueeze(0)
    a = L.MlpArgs()
    a.N, a.P, a.T = x.shape[1], theta.shape[1], theta.shape[0]
    if dx is None:
        dx = torch.empty_like(x)
    a.x, a.theta, a.dx, a.status = _p(x), _p(theta), _p(dx), _p(status)
    for k in MLP_KEYS:
        setattr(a, k, _p(w[k]))
    need = lib.avatar_mlp_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_mlp_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, x.device)
    L.check(lib.avatar_mlp(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_mlp")
    return dx


# ---------------------------------------------------------------- densification
def avatar_densify(knn, faces, xv, rand, d0=1.0, p0=0.02, out=None, ws=None, status=None, want_stats=False):
    """Alg. 1 (App. B): positions of the Gaussians to add.  knn [K_g, G]
    int32, faces [F, 3] int32, xv [3, N_v], rand [3, capacity] uniform words
    (int32 or uint32 storage).  Returns dict(count [1] device (N'), tri
    [capacity], x [3, capacity]) and, with want_stats, Dv, df, ng."""
    lib = L.load()
    ctx = context()
    dev = xv.device
    cap = rand.shape[1]
    a = L.DensifyArgs()
    a.G, a.Nv, a.F, a.Kg = knn.shape[1], xv.shape[1], faces.shape[0], knn.shape[0]
    a.knn, a.faces, a.xv = _p(knn), _p(faces), _p(xv)
    a.d0, a.p0, a.capacity = float(d0), float(p0), cap
    rand = rand.contiguous()
    if out is None:
        out = dict(count=torch.zeros(1, dtype=torch.int32, device=dev),
                   tri=torch.empty(cap, dtype=torch.int32, device=dev),
                   x=torch.empty(3, cap, dtype=torch.float32, device=dev))
        if want_stats:
            out.update(Dv=torch.empty(a.Nv, dtype=torch.int32, device=dev),
                       df=torch.empty(a.F, dtype=torch.float32, device=dev),
                       ng=torch.empty(a.F, dtype=torch.int32, device=dev))
    a.rand, a.count, a.tri, a.x = _p(rand), _p(out["count"]), _p(out["tri"]), _p(out["x"])
    a.Dv, a.df, a.ng, a.status = _p(out.get("Dv")), _p(out.get("df")), _p(out.get("ng")), _p(status)
    need = lib.avatar_densify_workspace_size(C.byref(a))
    if need == 0:
        raise L.AvatarError(1, "avatar_densify_workspace_size")
    if ws is None or ws.numel() < need:
        ws = workspace(need, dev)
    L.check(lib.avatar_densify(ctx, C.byref(a), _p(ws), ws.numel(), _stream()), "avatar_densify")
    return out


# ---------------------------------------------------------------- Adam
def avatar_adam(groups, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step over groups = [(param, grad, m, v, lr), ...] (contiguous
    tensors of equal element count; param float32 or bfloat16, the rest
    float32), updated in place; step t >= 1."""
    lib = L.load()
    ctx = context()
    if len(groups) > L.ADAM_MAX_GROUPS:
        raise ValueError(f"at most {L.ADAM_MAX_GROUPS} groups")
    a = L.AdamArgs()
    a.n_groups, a.beta1, a.beta2, a.eps, a.step = len(groups), beta1, beta2, eps, int(step)
    for k, (p, g, m, v, lr) in enumerate(groups):
        for x in (p, g, m, v):
            if not x.is_contiguous() or x.numel() != p.numel():
                raise ValueError("Adam tensors must be contiguous and of one size")
        gr = a.group[k]
        gr.n, gr.param, gr.grad, gr.m, gr.v, gr.lr = p.numel(), _p(p), _p(g), _p(m), _p(v), float(lr)
        gr.dtype = _dtype_code(p)
    L.check(lib.avatar_adam(ctx, C.byref(a), _stream()), "avatar_adam")


class Adam:
    """Adam state (FP32 moments) for named parameter tensors; step(grads)
    launches one fused update of every group."""

    def __init__(self, params, lr, beta1=0.9, beta2=0.999, eps=1e-15):
        self.params = params          # name -> tensor, updated in place
        self.lr = dict(lr)            # name -> learning rate
        self.b = (beta1, beta2, eps)
        self.m = {k: torch.zeros(p.shape, dtype=torch.float32, device=p.device) for k, p in params.items()}
        self.v = {k: torch.zeros(p.shape, dtype=torch.float32, device=p.device) for k, p in params.items()}
        self.t = 0

    def step(self, grads):
        self.t += 1
        groups = [(self.params[k], grads[k], self.m[k], self.v[k], self.lr[k]) for k in self.params]
        avatar_adam(groups, self.t, *self.b)


def probe_alu(kind, iters, sink):
    """Launches one pipe-throughput probe (avatar_probe_alu) on the current
    stream; returns the operations it executes.  kind: 'ffma', 'iadd3',
    'lop3' or 'imad'; sink: a 1-element int32 device tensor."""
    kinds = dict(ffma=L.PROBE_FFMA, iadd3=L.PROBE_IADD3, lop3=L.PROBE_LOP3, imad=L.PROBE_IMAD)
    ops = C.c_longlong(0)
    L.check(L.load().avatar_probe_alu(context(), kinds[kind], int(iters), _p(sink), C.byref(ops), _stream()),
            "avatar_probe_alu")
    return int(ops.value)


def gaussian_order(knn, Nv, status=None):
    """Stable order of the Gaussians by their nearest vertex (knn row 0)
    (avatar_gaussian_order); int32 [G]."""
    lib = L.load()
    _need_cuda(knn, "knn")
    G = knn.shape[-1]
    order = torch.empty(G, dtype=torch.int32, device=knn.device)
    ws = workspace(lib.avatar_gaussian_order_workspace_size(G), knn.device)
    nearest = knn[0] if knn.dim() == 2 else knn
    L.check(lib.avatar_gaussian_order(context(), G, int(Nv), _p(nearest), _p(order), _p(ws), ws.numel(), _p(status),
                                      _stream()), "avatar_gaussian_order")
    return order


def gather_columns(src, order, status=None):
    """dst[..., i] = src[..., order[i]] over the last dimension
    (avatar_gather_columns); src holds 2- or 4-byte elements.  A 3-d src
    [rows][n][m] of 4-byte elements (m <= 4) is gathered by its n records
    of m elements."""
    _need_cuda(src, "src")
    if src.dim() == 3:
        rows, n, m = src.shape
        elem = m * src.element_size()
    else:
        n = src.shape[-1]
        rows = src.numel() // max(n, 1)
        elem = src.element_size()
    if order.dim() != 1 or order.numel() != n:
        raise ValueError(f"order of {order.numel()} entries for {n} columns")
    dst = torch.empty_like(src)
    L.check(L.load().avatar_gather_columns(context(), rows, n, elem, _p(src), _p(dst), _p(order), _p(status),
                                           _stream()), "avatar_gather_columns")
    return dst
