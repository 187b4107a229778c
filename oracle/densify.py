"""Oracle of the density-based Gaussian densification (App. B, Alg. 1), in
FP64 and exact integers.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

Steps in the algorithm's order:
  D_v[k]  = number of Gaussians i with k in S_g^i            (integer)
  d_f[i]  = (sum of D_v over the three vertices of f^i) / (6 K_g)
  P[i]    = max(0, d0 - d_f[i])
  N'      = floor(sum(P) p0)
  n_g     = MultinomialSample(P / sum(P), N')
  n_g[i] Gaussians placed uniformly at random on triangle i.

Readings (the paper gives the steps, d0 = 1 and p0 = 0.02, nothing finer):
  * d0 6 K_g must be an integer (it is for d0 = 1); then
    P[i] = w[i] / (6 K_g) with the integer weight w[i] = max(0, d0 6 K_g - S_f[i]),
    sum(P) = W / (6 K_g), W = sum of w, and the sampling probabilities
    w[i] / W are exact.
  * N' = floor((p0 W) / (6 K_g)) evaluated in IEEE FP64 in that order (a
    fully specified value; it equals the exact floor of p0 sum(P) except when
    that product lies within FP64 rounding of an integer).
  * The random numbers are inputs: per draw j three uint32 values r0, r1, r2.
    Draw j selects the triangle t_j = the smallest i with cumsum(w)[i] > s_j,
    s_j = floor(r0 W / 2^32) (so t_j = i with probability w[i] / W up to the
    2^-32 granularity of r0); n_g[i] counts the draws that select i.
  * Placement of draw j on t_j = (a, b, c) of the canonical mesh: u = (r1 >> 8)
    2^-24, v = (r2 >> 8) 2^-24 (exact in FP32 and FP64); if u + v > 1 then
    (u, v) <- (1 - u, 1 - v); x = a + u (b - a) + v (c - a).  The added
    Gaussians are listed in draw order (the multiset of triangles is the
    multinomial sample n_g).
"""
from __future__ import annotations

import numpy as np


def vertex_counts(knn, nv):
    """D_v: for each vertex, how many Gaussians have it among their K_g nearest
    (knn [G, K_g])."""
    D = np.zeros(nv, np.int64)
    for row in np.asarray(knn, np.int64):
        for k in row:
            D[k] += 1
    return D


def densify(knn, faces, xv, rand, d0=1.0, p0=0.02):
    """Alg. 1.  knn [G, K_g], faces [F, 3], xv [N_v, 3] canonical vertices,
    rand [n, 3] uint32 (n >= the number of draws used).  Returns a dict with
    Dv, df, w, W, n_new, tri [n_new], ng [F], x [n_new, 3]."""
    knn = np.asarray(knn, np.int64)
    faces = np.asarray(faces, np.int64)
    xv = np.asarray(xv, np.float64)
    Kg = knn.shape[1]
    D = vertex_counts(knn, xv.shape[0])
    S = D[faces[:, 0]] + D[faces[:, 1]] + D[faces[:, 2]]
    df = S / (6.0 * Kg)
    thr = d0 * 6 * Kg
    if thr != int(thr):
        raise ValueError("d0 * 6 K_g must be an integer")
    w = np.maximum(0, int(thr) - S)
    W = int(w.sum())
    n_new = int(np.floor(np.float64(p0) * np.float64(W) / np.float64(6 * Kg))) if W > 0 else 0
    rand = np.asarray(rand, np.uint64)
    if n_new > rand.shape[0]:
        raise ValueError("not enough random numbers")
    cum = np.cumsum(w)
    tri = np.empty(n_new, np.int64)
    x = np.empty((n_new, 3))
    for j in range(n_new):
        s = (int(rand[j, 0]) * W) >> 32
        i = int(np.searchsorted(cum, s, side="right"))  # smallest i with cum[i] > s
        tri[j] = i
        u = float(int(rand[j, 1]) >> 8) * 2.0 ** -24
        v = float(int(rand[j, 2]) >> 8) * 2.0 ** -24
        if u + v > 1.0:
            u, v = 1.0 - u, 1.0 - v
        a, b, c = xv[faces[i]]
        x[j] = a + u * (b - a) + v * (c - a)
    ng = np.bincount(tri, minlength=faces.shape[0]).astype(np.int64)
    return dict(Dv=D, df=df, w=w, W=W, n_new=n_new, tri=tri, ng=ng, x=x)


__all__ = ["vertex_counts", "densify"]
