"""Frame-level composition of the four native stages.

Renderer   : the relit novel-pose frame (Sec. 3.1-3.2, test-time path of
             Sec. 3.5): skin -> visibility -> shade -> splat, all buffers
             preallocated so that a frame allocates nothing and can be
             captured in a CUDA graph.
TrainStep  : the differentiable step (Sec. 3.3): the frame above, the L1
             image loss and the hand-written backward kernels in reverse
             order (splat -> shade -> skin); also graph-capturable.
Autograd   : torch.autograd.Function wrappers of the same entry points for
             user training loops (visibility bits are constants, as the
             paper precomputes visibility for training poses, Sec. 3.5).

Only argument marshalling happens here; every arithmetic step is a kernel
of libavatar.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def scene_tensors(scene, device="cuda", attr_dtype="f32"):
    """Device copies of a synth.Scene (SoA float32 / int32; the learnable
    attributes in BF16 with attr_dtype='bf16')."""
    f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    t = api.avatar_tensors(scene.avatar, device, attr_dtype)
    light = dict(L=f(scene.light.L), A=f(scene.light.A), w=f(scene.light.w))
    return dict(avatar=t, light=light, frames=f(scene.frames.reshape(-1, 9)),
                dmap=torch.as_tensor(scene.dmap, dtype=torch.int32, device=device), camera=scene.camera,
                depth_res=int(scene.depth_res), center=[float(c) for c in scene.window_center],
                half=float(scene.window_half), bias=float(scene.vis_bias),
                cam_center=[float(c) for c in scene.camera.center])


GAUSSIAN_KEYS = ("xg", "logscale", "quat", "opacity", "knn")


def spatially_ordered(st, status=None):
    """The scene with its Gaussians stored in the order of their nearest
    vertex (avatar_gaussian_order, applied to every per-Gaussian array by
    avatar_gather_columns): a setup step, once per avatar, that lets the
    32 Gaussians of a warp share their neighbours' records.  Rendered images
    are the same (Gaussians of equal depth keys blend in index order, so a
    pixel can differ only where two depths tie exactly in FP32).  Returns
    (scene tensors, order): Gaussian i of the result is Gaussian order[i] of
    st."""
    t = st["avatar"]
    order = api.gaussian_order(t["knn"], t["xv"].shape[1], status)
    t2 = dict(t)
    for k in GAUSSIAN_KEYS:
        t2[k] = api.gather_columns(t[k], order, status)
    st2 = dict(st)
    st2["avatar"] = t2
    return st2, order


def faces_ordered(st, order, status=None):
    """The scene with its mesh faces stored in `order` (int32 [F], e.g.
    synth.face_normal_order, a permutation within the raster's chunks of
    _lib.VIS_FACE_CHUNK faces): the rows of faces [F][3] gathered by
    avatar_gather_columns.  The visibility bits, and so every image, are
    the same."""
    f = st["avatar"]["faces"]
    o = torch.as_tensor(np.ascontiguousarray(order, dtype=np.int32), device=f.device)
    if o.dim() != 1 or o.numel() != f.shape[0]:
        raise ValueError(f"face order of {o.numel()} entries for {f.shape[0]} faces")
    t2 = dict(st["avatar"])
    t2["faces"] = api.gather_columns(f.reshape(1, -1, 3), o, status).reshape(f.shape)
    st2 = dict(st)
    st2["avatar"] = t2
    return st2, o


def light_ordered(st, order, status=None):
    """The scene with its light texels stored in `order` (int32 [NL], e.g.
    synth.latlong_patch_order): radiance, solid angles, directions and the
    viewpoint map d(k) reordered by avatar_gather_columns, so the visibility
    bits and the shading's 32-light chunks follow it.  Texel s of the result
    is texel order[s] of st; the images are the same (the shading sums run
    in another order) and light gradients come back in the new order."""
    dev = st["light"]["L"].device
    o = torch.as_tensor(np.ascontiguousarray(order, dtype=np.int32), device=dev)
    lt = st["light"]
    if o.dim() != 1 or o.numel() != lt["A"].numel():
        raise ValueError(f"light order of {o.numel()} entries for {lt['A'].numel()} texels")
    st2 = dict(st)
    st2["light"] = dict(L=api.gather_columns(lt["L"].reshape(1, -1, 3), o, status).reshape(lt["L"].shape),
                        A=api.gather_columns(lt["A"], o, status),
                        w=api.gather_columns(lt["w"].reshape(1, -1, 3), o, status).reshape(lt["w"].shape))
    st2["dmap"] = api.gather_columns(st["dmap"], o, status)
    return st2, o


class Renderer:
    """Preallocated forward frame.  forward() launches exactly the library's
    kernels: on the current stream, except that with overlap (the default)
    cull, projection and binning run on a second stream forked after skinning
    and joined before the blend (same images).  vis_cull_back rasterises only light-facing
    triangles for visibility; it gives the same bits as the two-sided rule for
    closed, outward-wound meshes such as the capsule body (set it to False
    for open or inconsistently wound meshes).  shade_tc evaluates the shading
    sums on the tensor cores (BF16 weights, FP32 accumulation; needs a light
    count that is a multiple of 64).  mlp (weights from api.mlp_tensors)
    evaluates the pose-dependent displacement MLP of Sec. 3.1 on the canonical
    vertices before every skinning, in place of the avatar's fixed dxv."""

    def __init__(self, st, tile=16, pair_capacity=None, vis_cull_back=True, shade_tc=False, visibility="depth",
                 knn_v=None, rebind=False, mlp=None, overlap=True):
        self.st = st
        # overlap: after skinning, cull + project + bin run on a second
        # (high-priority) stream while visibility and shading run on the
        # calling one; the blend joins them (splatting needs only the cull
        # flags and, in the blend, the colours from shading)
        self.overlap = overlap
        self.mlp = mlp
        self.mlp_ws = None
        self.skin_t = st["avatar"]
        if mlp is not None:
            self.skin_t = dict(st["avatar"])
            self.skin_t["dxv"] = torch.empty_like(st["avatar"]["xv"])
            self.mlp_ws = api.workspace(api.mlp_workspace_size(st["avatar"]["xv"].shape[1],
                                                               st["avatar"]["pose"].numel()), st["avatar"]["xv"].device)
        # rebind: recompute each Gaussian's K nearest vertices (Eq. 1's S_g) on the
        # device before every frame, as the canonical positions may have moved
        self.rebind = rebind
        self.knn_ws = None
        self.vis_cull_back = vis_cull_back
        self.shade_tc = shade_tc
        self.tc_ws = None
        # visibility: "depth" = depth maps + per-vertex depth test (exact bits);
        # "paper" = the paper's triangle-ID images + median/median/mean filters over
        # the Kv nearest vertices knn_v ([Kv, Nv] int32, soft visibility)
        if visibility not in ("depth", "paper"):
            raise ValueError("visibility must be 'depth' or 'paper'")
        if visibility == "paper" and (knn_v is None or shade_tc):
            raise ValueError("the paper's visibility needs knn_v and the CUDA-core shading")
        self.visibility_mode = visibility
        self.knn_v = knn_v
        t = st["avatar"]
        dev = t["xg"].device
        self.device = dev
        self.status = api.status_word(dev)
        self.sk = api.alloc_skin_outputs(t)
        self.sk["_ws"] = None
        self.skin_ws = None
        G = t["xg"].shape[1]
        Nv = t["xv"].shape[1]
        NL = st["light"]["L"].shape[0]
        self.bits = torch.empty(Nv, (NL + 31) // 32, dtype=torch.int32, device=dev)
        self.vis_count = torch.empty(Nv, NL, dtype=torch.uint8, device=dev) if visibility == "paper" else None
        self.vis_ws = None
        self.sh = dict(color=torch.empty(3, G, device=dev), radiance=torch.empty(3, G, device=dev),
                       cull=torch.empty(G, dtype=torch.uint8, device=dev))
        self.sb = api.alloc_splat(G, st["camera"], tile, pair_capacity, dev)
        self.cull_b = torch.empty(G, dtype=torch.uint8, device=dev)  # the binning branch's cull flags
        self._side = torch.cuda.Stream(device=dev, priority=-1) if overlap else None
        self.graph = None
        # first eager call sizes the workspaces
        self.forward()
        torch.cuda.synchronize()

    def bind(self):
        t = self.st["avatar"]
        if self.knn_ws is None:
            import ctypes as C
            from . import _lib as L
            a = L.KnnArgs()
            a.N, a.M, a.K = t["xg"].shape[1], t["xv"].shape[1], t["knn"].shape[0]
            self.knn_ws = api.workspace(L.load().avatar_knn_workspace_size(C.byref(a)), self.device)
        api.avatar_knn(t["xg"], t["xv"], t["knn"].shape[0], out=t["knn"], ws=self.knn_ws, status=self.status)

    def skin(self):
        if self.rebind:
            self.bind()
        if self.mlp is not None:
            t = self.skin_t
            api.avatar_mlp(t["xv"], t["pose"].reshape(-1), self.mlp, dx=t["dxv"], ws=self.mlp_ws, status=self.status)
        out = api.avatar_skin(self.skin_t, out=self.sk, ws=self.skin_ws, status=self.status)
        self.skin_ws = out["_ws"]

    def visibility(self):
        st = self.st
        if self.visibility_mode == "paper":
            if self.vis_ws is None:
                self.vis_ws = self._vis_soft_ws()
            api.avatar_visibility_soft(self.sk["xp"], st["avatar"]["faces"], st["frames"], st["center"], st["half"],
                                       st["depth_res"], self.knn_v, dmap=st["dmap"], vis_count=self.vis_count,
                                       ws=self.vis_ws, status=self.status, cull_back=self.vis_cull_back)
            return
        if self.vis_ws is None:
            self.vis_ws = self._vis_ws()
        api.avatar_visibility(self.sk["xp"], st["avatar"]["faces"], st["frames"], st["center"], st["half"],
                              st["bias"], st["depth_res"], dmap=st["dmap"], bits=self.bits, ws=self.vis_ws,
                              status=self.status, cull_back=self.vis_cull_back)

    def _vis_soft_ws(self):
        import ctypes as C
        from . import _lib as L
        st = self.st
        a = L.VisSoftArgs()
        a.base = api._vis_struct(self.sk["xp"], st["avatar"]["faces"], st["frames"], st["center"], st["half"], 0.0,
                                 st["depth_res"], st["dmap"], None, None)
        a.Kv = self.knn_v.shape[0]
        return api.workspace(L.load().avatar_visibility_soft_workspace_size(C.byref(a)), self.device)

    def _vis_ws(self):
        import ctypes as C
        from . import _lib as L
        st = self.st
        a = api._vis_struct(self.sk["xp"], st["avatar"]["faces"], st["frames"], st["center"], st["half"],
                            st["bias"], st["depth_res"], st["dmap"], self.bits, None)
        return api.workspace(L.load().avatar_visibility_workspace_size(C.byref(a)), self.device)

    def shade(self):
        st = self.st
        if self.shade_tc:
            if self.tc_ws is None:
                self.tc_ws = self._tc_ws()
            L1 = st["light"]["L"].unsqueeze(0)
            api.avatar_shade_multi(self.sk, st["avatar"]["knn"], self.bits, st["light"], st["cam_center"], L1,
                                   out=self.sh["color"].unsqueeze(0), cull=self.sh["cull"], status=self.status,
                                   ws=self.tc_ws, radiance=self.sh["radiance"])
            return
        if self.visibility_mode == "paper":
            api.avatar_shade(self.sk, st["avatar"]["knn"], self.vis_count, st["light"], st["cam_center"], out=self.sh,
                             status=self.status, vis_den=self.knn_v.shape[0])
            return
        api.avatar_shade(self.sk, st["avatar"]["knn"], self.bits, st["light"], st["cam_center"], out=self.sh,
                         status=self.status)

    def _tc_ws(self):
        import ctypes as C
        from . import _lib as L
        m = L.ShadeMultiArgs()
        m.base.G = self.sk["xd"].shape[1]
        return api.workspace(L.load().avatar_shade_multi_workspace_size(C.byref(m)), self.device)

    def splat(self):
        t = self.st["avatar"]
        api.avatar_splat(self.sk["xd"], self.sk["cov"], t["opacity"], self.sh["color"], self.sh["cull"],
                         self.st["camera"], b=self.sb, status=self.status)

    def forward(self):
        self.skin()
        if not self.overlap:
            self.visibility()
            self.shade()
            self.splat()
            return self.sb.image
        t = self.st["avatar"]
        args = (self.sk["xd"], self.sk["cov"], t["opacity"], self.sh["color"], self.cull_b, self.st["camera"], self.sb,
                self.status)
        main, side = torch.cuda.current_stream(), self._side
        side.wait_stream(main)
        with torch.cuda.stream(side):
            api.avatar_cull(self.sk, self.st["cam_center"], cull=self.cull_b)
            api.avatar_splat_project(*args)
            api.avatar_splat_bin(*args)
        self.visibility()
        self.shade()
        main.wait_stream(side)
        api.avatar_splat_blend(*args)
        return self.sb.image

    def capture(self):
        """Capture forward() in a CUDA graph (after one eager call)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.forward()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.forward()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.sb.image

    def check(self):
        api.raise_on_status(self.status, "render")


# Adam learning rates per parameter group: 3DGS's defaults for the Gaussians
# (position, log-scale, rotation) and its colour rate for the materials; 3DGS
# steps opacity as a logit at 0.05, here it is stored directly, so the rate is
# scaled by the logistic slope at 1/2 (1/4); the LBS weights and the light are
# not in 3DGS (the paper gives no rates but the editing position rate 1.6e-6
# of Sec. 4).
ADAM_LR = dict(xg=1.6e-4, logscale=5e-3, quat=1e-3, opacity=1.25e-2, av=2.5e-3, rv=2.5e-3, pv=2.5e-3, wv=1e-3,
               L=1e-2)


class TrainStep(Renderer):
    """Forward frame + image loss + backward through every stage; update()
    applies one fused Adam step to every trainable tensor (adam=True for
    ADAM_LR, or a dict of rates)."""

    def __init__(self, st, target, tile=16, pair_capacity=None, vis_cull_back=True, shade_tc=False,
                 visibility="depth", knn_v=None, rebind=False, ssim_weight=0.2, regularize=False, adam=None):
        # image loss of Eq. 5: (1 - ssim_weight) L1 + ssim_weight D-SSIM (the paper's 0.2);
        # regularize adds the regularisers of Sec. 3.3 (needs knn_v, the filters' S_v)
        self.target = target
        self.ssim_weight = float(ssim_weight)
        self.loss_ws = None
        if regularize and knn_v is None:
            raise ValueError("the smoothness regulariser needs knn_v")
        self.regularize = regularize
        self.reg_ws = None
        self.reg_terms = None
        super().__init__(st, tile, pair_capacity, vis_cull_back, shade_tc, visibility, knn_v, rebind)
        t = st["avatar"]
        self.loss = torch.empty(1, device=self.device)
        self.d_img = torch.empty_like(self.sb.image)
        self.g_splat = dict(xd=torch.empty_like(self.sk["xd"]), cov=torch.empty_like(self.sk["cov"]),
                            opacity=torch.empty_like(t["opacity"], dtype=torch.float32),
                            color=torch.empty_like(self.sh["color"]))
        self.g_shade = dict(xd=torch.empty_like(self.sk["xd"]), nd=torch.empty_like(self.sk["nd"]),
                            ag=torch.empty_like(self.sk["ag"]), rg=torch.empty_like(self.sk["rg"]),
                            pg=torch.empty_like(self.sk["pg"]), ubar=torch.empty_like(self.sk["ubar"]),
                            L=torch.empty_like(st["light"]["L"]))
        self.g_skin = {k: torch.empty_like(t[k], dtype=torch.float32)
                       for k in ("xg", "logscale", "quat", "wv", "av", "rv", "pv")}
        self._bwd_ws = None
        self.opt = None
        if adam:
            lr = ADAM_LR if adam is True else adam
            params = {k: t[k] for k in ("xg", "logscale", "quat", "opacity", "wv", "av", "rv", "pv")}
            params["L"] = st["light"]["L"]
            self.opt = api.Adam(params, lr)
        self.step()
        torch.cuda.synchronize()

    def backward(self):
        import ctypes as C
        from . import _lib as L
        lib = L.load()
        ctx = api.context()
        st = self.st
        t = st["avatar"]
        s = api._stream()
        # loss
        if self.loss_ws is None:
            la = L.ImageLossArgs()
            la.C, la.H, la.W = self.sb.image.shape
            la.lam, la.weight = self.ssim_weight, 1.0
            self.loss_ws = api.workspace(lib.avatar_image_loss_workspace_size(C.byref(la)), self.device)
        api.avatar_image_loss(self.sb.image, self.target, self.ssim_weight, d_img=self.d_img, loss=self.loss,
                              ws=self.loss_ws)
        # splat adjoint
        G = t["xg"].shape[1]
        a = api._splat_struct(G, st["camera"], self.sk["xd"], self.sk["cov"], t["opacity"], self.sh["color"],
                              self.sh["cull"], self.sb, None)
        gs = L.SplatGrads()
        gs.d_image = api._p(self.d_img)
        gs.d_xd, gs.d_cov, gs.d_opacity, gs.d_color = (api._p(self.g_splat[k]) for k in
                                                       ("xd", "cov", "opacity", "color"))
        L.check(lib.avatar_splat_backward(ctx, C.byref(a), C.byref(gs), api._p(self.sb.ws), self.sb.ws.numel(), s),
                "avatar_splat_backward")
        # shade adjoint
        if self.visibility_mode == "paper":
            sa = api._shade_struct(self.sk, t["knn"], self.vis_count, st["light"], st["cam_center"], self.sh["color"],
                                   self.sh["radiance"], self.sh["cull"], None, vis_den=self.knn_v.shape[0])
        else:
            sa = api._shade_struct(self.sk, t["knn"], self.bits, st["light"], st["cam_center"], self.sh["color"],
                                   self.sh["radiance"], self.sh["cull"], None)
        gh = L.ShadeGrads()
        gh.d_color = api._p(self.g_splat["color"])
        gh.d_xd, gh.d_nd, gh.d_ag, gh.d_rg, gh.d_pg, gh.d_ubar, gh.d_light_L = (
            api._p(self.g_shade[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar", "L"))
        L.check(lib.avatar_shade_backward(ctx, C.byref(sa), C.byref(gh), s), "avatar_shade_backward")
        # skin adjoint
        ka = api._skin_struct(t, self.sk, None)
        gk = L.SkinGrads()
        gk.d_xd, gk.d_xd2 = api._p(self.g_splat["xd"]), api._p(self.g_shade["xd"])
        gk.d_cov, gk.d_nd = api._p(self.g_splat["cov"]), api._p(self.g_shade["nd"])
        gk.d_ag, gk.d_rg, gk.d_pg, gk.d_ubar = (api._p(self.g_shade[k]) for k in ("ag", "rg", "pg", "ubar"))
        for k in ("xg", "logscale", "quat", "wv", "av", "rv", "pv"):
            setattr(gk, "d_" + k, api._p(self.g_skin[k]))
        if self._bwd_ws is None:
            self._bwd_ws = api.workspace(lib.avatar_skin_backward_workspace_size(C.byref(ka)), self.device)
        L.check(lib.avatar_skin_backward(ctx, C.byref(ka), C.byref(gk), api._p(self.skin_ws), api._p(self._bwd_ws),
                                         self._bwd_ws.numel(), s), "avatar_skin_backward")
        if self.regularize:
            if self.reg_ws is None:
                self.reg_ws = api.workspace(1 << 16, self.device)
                self.reg_terms = torch.zeros(4, device=self.device)
            api.avatar_regularizers(t, self.knn_v, grads=self.g_skin, loss=self.loss, terms=self.reg_terms,
                                    accumulate=True, ws=self.reg_ws, status=self.status)

    def step(self):
        self.forward()
        self.backward()
        return self.loss

    def update(self):
        """One Adam step on the gradients of the last step()."""
        self.opt.step(self.grads())

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self.graph = g
        return g

    def grads(self):
        return dict(**self.g_skin, opacity=self.g_splat["opacity"], L=self.g_shade["L"])


# ---------------------------------------------------------------- autograd
class SkinFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xg, logscale, quat, wv, av, rv, pv, const):
        t = dict(const)
        t.update(xg=xg.detach(), logscale=logscale.detach(), quat=quat.detach(), wv=wv.detach(), av=av.detach(),
                 rv=rv.detach(), pv=pv.detach())
        out = api.avatar_skin(t)
        ctx.t = t
        ctx.out = out
        ctx.mark_non_differentiable(out["xp"])
        return out["xp"], out["xd"], out["cov"], out["nd"], out["ag"], out["rg"], out["pg"], out["ubar"]

    @staticmethod
    def backward(ctx, dxp, dxd, dcov, dnd, dag, drg, dpg, dubar):
        up = dict(d_xd=dxd, d_cov=dcov, d_nd=dnd, d_ag=dag, d_rg=drg, d_pg=dpg, d_ubar=dubar)
        g = api.avatar_skin_backward(ctx.t, ctx.out, up)
        return g["xg"], g["logscale"], g["quat"], g["wv"], g["av"], g["rv"], g["pv"], None


class ShadeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xd, nd, ag, rg, pg, ubar, L, const):
        sk = dict(xd=xd.detach(), nd=nd.detach(), ag=ag.detach(), rg=rg.detach(), pg=pg.detach(),
                  ubar=ubar.detach())
        light = dict(L=L.detach(), A=const["A"], w=const["w"])
        out = api.avatar_shade(sk, const["knn"], const["bits"], light, const["cam_center"])
        ctx.sk, ctx.light, ctx.const, ctx.out = sk, light, const, out
        ctx.mark_non_differentiable(out["cull"])
        return out["color"], out["cull"]

    @staticmethod
    def backward(ctx, dcolor, dcull):
        c = ctx.const
        g = api.avatar_shade_backward(ctx.sk, c["knn"], c["bits"], ctx.light, c["cam_center"], ctx.out, dcolor)
        return g["xd"], g["nd"], g["ag"], g["rg"], g["pg"], g["ubar"], g["L"], None


class SplatFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xd, cov, opacity, color, cull, cam, tile=16):
        xd, cov, opacity, color = xd.detach(), cov.detach(), opacity.detach(), color.detach()
        b = api.avatar_splat(xd, cov, opacity, color, cull, cam, tile=tile)
        ctx.saved = (xd, cov, opacity, color, cull, cam, b)
        return b.image

    @staticmethod
    def backward(ctx, dimg):
        xd, cov, opacity, color, cull, cam, b = ctx.saved
        g = api.avatar_splat_backward(xd, cov, opacity, color, cull, cam, b, dimg)
        return g["xd"], g["cov"], g["opacity"], g["color"], None, None, None


class L1Fn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, target):
        loss, d = api.avatar_l1_loss(img.detach(), target)
        ctx.save_for_backward(d)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (d,) = ctx.saved_tensors
        return d * g, None


def render_differentiable(params, st, bits, tile=16):
    """One frame through the autograd wrappers.  params: leaf tensors xg,
    logscale, quat, opacity, wv, av, rv, pv, L (device layout)."""
    t = st["avatar"]
    const = {k: t[k] for k in ("knn", "xv", "dxv", "nv", "parents", "joints", "pose")}
    xp, xd, cov, nd, ag, rg, pg, ub = SkinFn.apply(params["xg"], params["logscale"], params["quat"], params["wv"],
                                                   params["av"], params["rv"], params["pv"], const)
    sconst = dict(A=st["light"]["A"], w=st["light"]["w"], knn=t["knn"], bits=bits, cam_center=st["cam_center"])
    color, cull = ShadeFn.apply(xd, nd, ag, rg, pg, ub, params["L"], sconst)
    return SplatFn.apply(xd, cov.reshape(6, -1), params["opacity"], color, cull, st["camera"], tile)


# ---------------------------------------------------------------- batching
class BatchRenderer:
    """Many poses (each with its own light) and cameras of mixed resolution
    rendered by avatar_render_batch: one launch per stage for the whole
    batch, capturable in one CUDA graph.  step() adds the L1 loss over all
    views' pixels and the batched backward (avatar_render_batch_backward).

    batch: a synth.Batch; attr_dtype 'bf16' stores the learnable attributes
    in BF16; spatial_order stores the Gaussians in the order of their
    nearest vertex (as spatially_ordered; self.order then maps Gaussian i
    to the batch avatar's Gaussian self.order[i]); light_order (int32 [NL])
    stores every pose's light texels in that order (as light_ordered);
    face_order (int32 [F]) stores the mesh faces in that order (as
    faces_ordered).  The pair buffer grows once if the first eager call
    overflows."""

    def __init__(self, batch, targets=None, tile=0, pair_capacity=None, vis_cull_back=True, attr_dtype="f32",
                 device="cuda", ssim_weight=0.2, spatial_order=False, light_order=None, face_order=None):
        import ctypes as C
        from . import _lib as L
        self.L, self.C = L, C
        sc = batch.scene
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
        self.t = api.avatar_tensors(sc.avatar, device, attr_dtype)
        self.order = None
        if spatial_order:
            st, self.order = spatially_ordered({"avatar": self.t})
            self.t = st["avatar"]
        if face_order is not None:
            self.t = faces_ordered({"avatar": self.t}, face_order)[0]["avatar"]
        self.frames = f(sc.frames.reshape(-1, 9))
        self.light_A, self.light_w = f(sc.light.A), f(sc.light.w)
        self.dmap = torch.as_tensor(sc.dmap, dtype=torch.int32, device=device)
        self.poses = f(batch.poses)
        self.light_L = f(batch.lights)
        self.B, self.V = batch.B, batch.V
        self.light_order = None
        if light_order is not None:
            # every pose's light texels, their geometry and d(k) in the given order (as light_ordered)
            o = torch.as_tensor(np.ascontiguousarray(light_order, dtype=np.int32), device=device)
            self.light_L = api.gather_columns(self.light_L, o)
            self.light_A = api.gather_columns(self.light_A, o)
            self.light_w = api.gather_columns(self.light_w.reshape(1, -1, 3), o).reshape(self.light_w.shape)
            self.dmap = api.gather_columns(self.dmap, o)
            self.light_order = o
        self.cameras = list(batch.cameras)
        self.view_pose = np.asarray(batch.view_pose, np.int32)
        self.sizes = [(c.height, c.width) for c in self.cameras]
        self.offsets = np.concatenate([[0], np.cumsum([3 * h * w for h, w in self.sizes])]).astype(np.int64)
        self.images = torch.empty(int(self.offsets[-1]), device=device)
        self.num_pairs = torch.zeros(1, dtype=torch.int32, device=device)
        self.status = api.status_word(device)
        self.device = device
        self.views = (L.View * self.V)()
        for v, cam in enumerate(self.cameras):
            self.views[v].cam = api.camera_struct(cam)
            self.views[v].pose = int(self.view_pose[v])
            for k in range(3):
                self.views[v].center[k] = float(cam.center[k])
        G = self.t["xg"].shape[1]
        self.G = G
        self.tile = int(tile)
        self.cull_back = vis_cull_back
        self.sc = sc
        cap = pair_capacity or min(0x7FFFFFFF, max(65536, 16 * G * self.V))
        self._alloc(cap)
        self.targets = targets
        self.ssim_weight = float(ssim_weight)
        self.graph = None
        self.forward()
        torch.cuda.synchronize()
        need = int(self.num_pairs.item())
        if pair_capacity is None and need > cap:
            self._alloc(min(0x7FFFFFFF, int(need * 1.25) + 1024))
            self.status.zero_()
            self.forward()
            torch.cuda.synchronize()
        self.check()
        if targets is not None:
            self._alloc_grads()
            self.step()
            torch.cuda.synchronize()
            self.check()

    def _desc(self):
        L = self.L
        d = L.BatchDesc()
        t = self.t
        d.avatar = api._skin_struct(t, dict(bone=None, xp=None, xd=None, cov=None, nd=None, ag=None, rg=None,
                                            pg=None, ubar=None), None)
        d.opacity = api._p(t["opacity"])
        d.F = t["faces"].shape[0]
        d.faces = api._p(t["faces"])
        d.D = self.frames.shape[0]
        d.R = int(self.sc.depth_res)
        d.frames = api._p(self.frames)
        for k in range(3):
            d.center[k] = float(self.sc.window_center[k])
        d.half_extent = float(self.sc.window_half)
        d.bias = float(self.sc.vis_bias)
        d.cull_back = 1 if self.cull_back else 0
        d.NL = self.light_A.shape[0]
        d.light_A, d.light_w, d.dmap = api._p(self.light_A), api._p(self.light_w), api._p(self.dmap)
        d.B = self.B
        d.poses = api._p(self.poses)
        d.light_L = api._p(self.light_L)
        d.V = self.V
        d.views = self.C.cast(self.views, self.C.c_void_p)
        d.tile = self.tile
        d.pair_capacity = self.cap
        d.images = api._p(self.images)
        d.num_pairs = api._p(self.num_pairs)
        d.status = api._p(self.status)
        return d

    def _alloc(self, cap):
        self.cap = int(cap)
        self.ws = None
        d = self._desc()
        need = self.L.load().avatar_render_batch_workspace_size(self.C.byref(d))
        if need == 0:
            raise self.L.AvatarError(1, "avatar_render_batch_workspace_size")
        self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)

    def _alloc_grads(self):
        t = self.t
        e = lambda k: torch.empty_like(t[k], dtype=torch.float32)
        self.grads = dict(xg=e("xg"), logscale=e("logscale"), quat=e("quat"), opacity=e("opacity"), wv=e("wv"),
                          av=e("av"), rv=e("rv"), pv=e("pv"), L=torch.empty_like(self.light_L))
        self.loss = torch.empty(1, device=self.device)
        self.d_images = torch.empty_like(self.images)

    def _gstruct(self, d_images):
        g = self.L.BatchGrads()
        g.d_images = api._p(d_images)
        for k in ("xg", "logscale", "quat", "opacity", "wv", "av", "rv", "pv"):
            setattr(g, "d_" + k, api._p(self.grads[k]))
        g.d_light_L = api._p(self.grads["L"])
        return g

    def image(self, v):
        h, w = self.sizes[v]
        return self.images[self.offsets[v]:self.offsets[v + 1]].view(3, h, w)

    def forward(self):
        d = self._desc()
        self.L.check(self.L.load().avatar_render_batch(api.context(), self.C.byref(d), api._p(self.ws),
                                                        self.ws.numel(), api._stream()), "avatar_render_batch")
        return self.images

    def backward(self, d_images):
        d = self._desc()
        g = self._gstruct(d_images)
        self.L.check(self.L.load().avatar_render_batch_backward(api.context(), self.C.byref(d), self.C.byref(g),
                                                                 api._p(self.ws), self.ws.numel(), api._stream()),
                     "avatar_render_batch_backward")
        return self.grads

    def step(self):
        """Forward, the image loss of Eq. 5 over every view (each view's loss
        weighted by its share of all pixels), backward."""
        self.forward()
        total = float(self.offsets[-1])
        if getattr(self, "loss_ws", None) is None:
            la = self.L.ImageLossArgs()
            h, w = max(self.sizes, key=lambda s: s[0] * s[1])
            la.C, la.H, la.W, la.lam, la.weight = 3, h, w, self.ssim_weight, 1.0
            self.loss_ws = api.workspace(self.L.load().avatar_image_loss_workspace_size(self.C.byref(la)),
                                         self.device)
        for v, (h, w) in enumerate(self.sizes):
            sl = slice(int(self.offsets[v]), int(self.offsets[v + 1]))
            api.avatar_image_loss(self.images[sl].view(3, h, w), self.targets[sl].view(3, h, w), self.ssim_weight,
                                  d_img=self.d_images[sl].view(3, h, w), loss=self.loss, ws=self.loss_ws,
                                  weight=3 * h * w / total, accumulate=v > 0)
        self.backward(self.d_images)
        return self.loss

    def autotune(self, with_grads=None):
        """Runs the library's autotuner on this batch; returns (tile, ppt, bwd_ppt)."""
        with_grads = self.targets is not None if with_grads is None else with_grads
        d = self._desc()
        tuned = (self.C.c_int * 3)()
        g = self._gstruct(self.d_images) if with_grads else None
        self.L.check(self.L.load().avatar_render_batch_autotune(
            api.context(), self.C.byref(d), self.C.byref(g) if g is not None else None, api._p(self.ws),
            self.ws.numel(), api._stream(), tuned), "avatar_render_batch_autotune")
        return tuple(tuned)

    def capture(self, train=None):
        """Capture forward() (or step() with train=True) in one CUDA graph."""
        train = self.targets is not None if train is None else train
        fn = self.step if train else self.forward
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.images

    def check(self):
        api.raise_on_status(self.status, "render_batch")


def densify(st, rand, d0=1.0, p0=0.02, logscale=-4.0, opacity=0.5, status=None):
    """Alg. 1 (App. B) on the avatar of st: appends the Gaussians it places
    (positions from the device; log-scale `logscale` on every axis, the
    identity rotation, opacity `opacity`) and recomputes every Gaussian's K_g
    nearest vertices (S_g of Eq. 1).  rand: [3, capacity] uniform 32-bit words.
    Returns the number added.  A training-control step (the paper runs it every
    100 iterations): it reads the count back to grow the tensors, and the
    renderers built on st must be rebuilt."""
    t = st["avatar"]
    out = api.avatar_densify(t["knn"], t["faces"], t["xv"], rand, d0, p0, status=status)
    n = min(int(out["count"].item()), rand.shape[1])
    if n == 0:
        return 0
    dev = t["xg"].device
    t["xg"] = torch.cat([t["xg"], out["x"][:, :n]], 1).contiguous()
    t["logscale"] = torch.cat([t["logscale"], torch.full((3, n), logscale, dtype=t["logscale"].dtype, device=dev)],
                              1).contiguous()
    q = torch.zeros(4, n, dtype=t["quat"].dtype, device=dev)
    q[0] = 1.0
    t["quat"] = torch.cat([t["quat"], q], 1).contiguous()
    t["opacity"] = torch.cat([t["opacity"], torch.full((n,), opacity, dtype=t["opacity"].dtype, device=dev)])
    t["knn"] = api.avatar_knn(t["xg"], t["xv"], t["knn"].shape[0], status=status)
    return n


def average_displacement(st, mlp, poses, status=None):
    """Sec. 4's displacement for novel poses: the mean of the MLP's
    displacement over the training poses (poses [T, 72], weights from
    api.mlp_tensors), stored as the avatar's fixed displacement dxv."""
    t = st["avatar"]
    api.avatar_mlp(t["xv"], poses.reshape(poses.shape[0], -1), mlp, dx=t["dxv"], status=status)
    return t["dxv"]
