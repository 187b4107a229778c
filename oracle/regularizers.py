"""FP64 oracle of the training regularisers of Sec. 3.3 (the terms of Eq. 6
beside the image loss).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

  L_smooth = sum_i sum_{k in S_v^i} ( |a_i - a_k|_1 + |gamma_i - gamma_k| + |p_i - p_k| )
  L_mdist  = sum_i sum_{k in S_g^i} || x_g^i - x_v^k ||_2
  L_disp   = sum_i || dx^i ||_2
  L_scale  = sum_i sum_c max(0, s_g^{i,c} - s0),  s_g = exp(log-scale)
  L_reg    = w_smooth L_smooth + w_mdist L_mdist + w_disp L_disp + w_scale L_scale
(paper: w = 0.002, 0.1, 0.02, 10 and s0 = 0.005).  The gradient is FP64
autograd of the same expressions; |.| and ||.|| take the subgradient 0 at 0.
"""
from __future__ import annotations

import numpy as np

WEIGHTS = dict(smooth=0.002, mdist=0.1, disp=0.02, scale=10.0)
S0 = 0.005


def terms_torch(xg, logscale, knn, xv, av, rv, pv, knn_v, dxv, s0=S0):
    """The four unweighted sums on FP64 torch tensors in the oracle's AoS
    layout (xg [G,3], logscale [G,3], knn [G,Kg], xv [Nv,3], av [Nv,3],
    rv [Nv], pv [Nv], knn_v [Nv,Kv], dxv [Nv,3])."""
    import torch
    kv = torch.as_tensor(np.asarray(knn_v, np.int64))
    kg = torch.as_tensor(np.asarray(knn, np.int64))
    smooth = ((av[:, None, :] - av[kv]).abs().sum() + (rv[:, None] - rv[kv]).abs().sum()
              + (pv[:, None] - pv[kv]).abs().sum())
    mdist = torch.linalg.vector_norm(xg[:, None, :] - xv[kg], dim=-1).sum()
    disp = torch.linalg.vector_norm(dxv, dim=-1).sum()
    scale = torch.clamp(torch.exp(logscale) - s0, min=0.0).sum()
    return dict(smooth=smooth, mdist=mdist, disp=disp, scale=scale)


def regularizers(xg, logscale, knn, xv, av, rv, pv, knn_v, dxv, weights=None, s0=S0):
    """(total, terms, grads) with grads for xg, logscale, av, rv, pv, dxv."""
    import torch
    w = dict(WEIGHTS if weights is None else weights)
    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True)
         for k, v in dict(xg=xg, logscale=logscale, av=av, rv=rv, pv=pv, dxv=dxv).items()}
    xv_t = torch.tensor(np.asarray(xv, np.float64))
    terms = terms_torch(t["xg"], t["logscale"], knn, xv_t, t["av"], t["rv"], t["pv"], knn_v, t["dxv"], s0)
    total = sum(w[k] * terms[k] for k in terms)
    total.backward()
    grads = {k: (v.grad.numpy() if v.grad is not None else np.zeros(v.shape)) for k, v in t.items()}
    return float(total), {k: float(v) for k, v in terms.items()}, grads


__all__ = ["WEIGHTS", "S0", "terms_torch", "regularizers"]
