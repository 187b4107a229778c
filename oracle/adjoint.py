"""FP64 analytic adjoint of the differentiable render path, by PyTorch CPU
autograd over a plain restatement of the forward definitions.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU leg).  It is a
second, independent writing of the forward pass of avatar_oracle.c in torch
float64 (skinning: Sec. 3.1 / Eq. 1; shading: Eq. 2 + App. A; EWA projection
and front-to-back compositing: the 3DGS rasteriser of Sec. 3.1; L1 image loss:
Eq. 5).  Its forward must agree with the C oracle and its gradient with
central finite differences of the C oracle; both are checked in
tests/test_oracle_pins.py.  Visibility bits enter as constants (the paper
precomputes visibility for training poses, Sec. 3.5).

Compositing is written for all pixels at once: every pixel sees the same
(depth, index) order, so the per-pixel sorted list is the global order
filtered by alpha >= 1/255, and the front-to-back stop rule becomes a
cumulative mask.
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


def t64(a):
    return torch.as_tensor(np.asarray(a), dtype=DT)


def quat_to_rot(q):
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=-1).reshape(*q.shape[:-1], 3, 3)


def skin(xg, logscale, quat, knn, xv, dxv, wv, av, rv, pv, nv, bone):
    """Eq. 1 interpolation + LBS (Sec. 3.1). bone: [J,3,4]."""
    knn = torch.as_tensor(knn, dtype=torch.long)
    xj = xv[knn]                                            # [G,K,3]
    d = (xg[:, None, :] - xj).norm(dim=-1)
    u = 1.0 / torch.clamp(d, min=1e-8)
    ub = u / u.sum(dim=1, keepdim=True)                     # [G,K]
    interp = lambda t: torch.einsum("gk,gk...->g...", ub, t[knn])
    ag, rg, pg = interp(av), interp(rv), interp(pv)
    ng = interp(nv)
    wg = interp(wv)
    dxg = interp(dxv)
    A = torch.einsum("gj,jab->gab", wg, bone)               # [G,3,4]
    M, tr = A[:, :, :3], A[:, :, 3]
    xb = xg + dxg
    xd = torch.einsum("gab,gb->ga", M, xb) + tr
    R = quat_to_rot(quat)
    S = R * torch.exp(2.0 * logscale)[:, None, :]
    Sigma = S @ R.transpose(1, 2)
    cov = M @ Sigma @ M.transpose(1, 2)
    ng = ng / ng.norm(dim=-1, keepdim=True)
    m = torch.einsum("gab,gb->ga", M, ng)
    nd = m / m.norm(dim=-1, keepdim=True)
    return dict(xd=xd, cov=cov, nd=nd, ag=ag, rg=rg, pg=pg, ubar=ub, wg=wg)


def vis_matrix(ubar, knn, bits, dmap):
    """vis[g,k] = sum_j ubar_gj bit(S_gj, d(k)) (Eq. 1 applied to v)."""
    knn = np.asarray(knn)
    dmap = np.asarray(dmap)
    words = bits[knn][:, :, dmap >> 5]                      # [G,K,NL]
    b = ((words >> (dmap & 31).astype(np.uint32)) & 1).astype(np.float64)
    return torch.einsum("gj,gjk->gk", ubar, t64(b))


def shade(xd, nd, ag, rg, pg, vis, L, A, w, cam_center, culled):
    """Eq. 2 with the BRDF of App. A; returns colour [G,3] (culled -> 0)."""
    wo = cam_center[None, :] - xd
    wo = wo / wo.norm(dim=-1, keepdim=True)
    co = torch.clamp((nd * wo).sum(-1), min=0.0)            # [G]
    ci = nd @ w.T                                            # [G,NL]
    lit = (ci > 0).to(DT) * (vis > 0).to(DT)
    h = w[None, :, :] + wo[:, None, :]
    h = h / torch.clamp(h.norm(dim=-1, keepdim=True), min=1e-30)
    nh = torch.einsum("gc,gkc->gk", nd, h)
    voh = torch.einsum("gc,gkc->gk", wo, h)
    alpha = rg * rg
    a2 = (alpha * alpha)[:, None]
    kk = ((rg + 1.0) ** 2 / 8.0)[:, None]
    den = nh * nh * (a2 - 1.0) + 1.0
    Dn = a2 / (math.pi * den * den)
    Fr = 0.04 + 0.96 * torch.pow(2.0, (-5.55473 * voh - 6.98316) * voh)
    cic = torch.clamp(ci, min=0.0)
    fs = Dn * Fr / (4.0 * (cic * (1.0 - kk) + kk) * (co[:, None] * (1.0 - kk) + kk))
    wgt = lit * vis * cic                                    # [G,NL]
    B = L * A[:, None]                                       # [NL,3]
    diffuse = (wgt @ B) * ag / math.pi
    spec = ((wgt * fs) @ B) * pg[:, None]
    Lo = diffuse + spec
    col = torch.pow(torch.clamp(Lo, min=1e-6), 1.0 / 2.2)
    keep = (~torch.as_tensor(np.asarray(culled, bool)))[:, None].to(DT)
    return col * keep


def project(xd, cov, cam):
    R = t64(cam.R)
    t = t64(cam.t)
    p = xd @ R.T + t
    x, y, z = p.unbind(-1)
    mean2d = torch.stack([cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy], dim=-1)
    zero = torch.zeros_like(z)
    Jm = torch.stack([torch.stack([cam.fx / z, zero, -cam.fx * x / (z * z)], -1),
                      torch.stack([zero, cam.fy / z, -cam.fy * y / (z * z)], -1)], dim=1)
    T = Jm @ R
    S2 = T @ cov @ T.transpose(1, 2)
    s00 = S2[:, 0, 0] + 0.3
    s01 = S2[:, 0, 1]
    s11 = S2[:, 1, 1] + 0.3
    det = s00 * s11 - s01 * s01
    conic = torch.stack([s11 / det, -s01 / det, s00 / det], dim=-1)
    return mean2d, conic, z


def composite(mean2d, conic, opacity, color, depth, valid, width, height):
    """Front-to-back blending of all valid Gaussians at every pixel centre."""
    valid = np.asarray(valid).astype(bool)
    idx = np.nonzero(valid)[0]
    dnp = depth.detach().numpy()[idx]
    order = idx[np.lexsort((idx, dnp))]
    o = torch.as_tensor(order, dtype=torch.long)
    m, c, op, col = mean2d[o], conic[o], opacity[o], color[o]
    ys, xs = torch.meshgrid(torch.arange(height, dtype=DT) + 0.5,
                            torch.arange(width, dtype=DT) + 0.5, indexing="ij")
    px = xs.reshape(-1, 1)
    py = ys.reshape(-1, 1)
    dx = px - m[None, :, 0]
    dy = py - m[None, :, 1]
    q = c[None, :, 0] * dx * dx + 2.0 * c[None, :, 1] * dx * dy + c[None, :, 2] * dy * dy
    araw = op[None, :] * torch.exp(-0.5 * q)
    a = torch.clamp(araw, max=0.99)
    mask = (a.detach() >= 1.0 / 255.0)
    am = a * mask.to(DT)
    Tin = torch.cumprod(1.0 - am.detach(), dim=1)
    stop = mask & (Tin < 1e-4)
    inc = mask & (torch.cumsum(stop.to(torch.int64), dim=1) == 0)
    ai = a * inc.to(DT)
    ones = torch.ones(ai.shape[0], 1, dtype=DT)
    Tex = torch.cat([ones, torch.cumprod(1.0 - ai, dim=1)[:, :-1]], dim=1)
    w = ai * Tex
    img = w @ col                                            # [P,3]
    return img.reshape(height, width, 3)


def render(params, fixed, return_parts=False):
    """Whole differentiable frame. params: dict of leaf tensors (xg, logscale,
    quat, opacity, av, rv, pv, L, wv); fixed: dict of constants."""
    sk = skin(params["xg"], params["logscale"], params["quat"], fixed["knn"], fixed["xv"],
              fixed["dxv"], params["wv"], params["av"], params["rv"], params["pv"], fixed["nv"],
              fixed["bone"])
    vis = vis_matrix(sk["ubar"], fixed["knn"], fixed["bits"], fixed["dmap"])
    col = shade(sk["xd"], sk["nd"], sk["ag"], sk["rg"], sk["pg"], vis, params["L"], fixed["A"],
                fixed["w"], fixed["cam_center"], fixed["culled"])
    mean2d, conic, depth = project(sk["xd"], sk["cov"], fixed["cam"])
    img = composite(mean2d, conic, params["opacity"], col, depth, fixed["valid"],
                    fixed["cam"].width, fixed["cam"].height)
    if return_parts:
        return img, dict(sk=sk, vis=vis, col=col, mean2d=mean2d, conic=conic, depth=depth)
    return img


def l1_loss(img, target):
    """Mean absolute error over pixels and channels (L1 part of Eq. 5)."""
    return (img - target).abs().mean()
