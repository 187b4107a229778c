"""FP64 oracle of the pose-dependent displacement MLP (Sec. 3.1; its design
in Sec. 4: four layers of width 256 with ReLU, Random Fourier Features of the
coordinates): dx = d(x, theta).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

Reading (the paper gives the layer count, width, activation and the use of
random Fourier features, not the feature count or the layer layout):
  gamma(x) = [sin(2 pi B x), cos(2 pi B x)]            B: [64, 3] frequencies
  z1 = W1 [gamma(x); theta] + b1,   h1 = relu(z1)        W1: [256, 128 + P]
  h2 = relu(W2 h1 + b2),  h3 = relu(W3 h2 + b3)          W2, W3: [256, 256]
  dx = W4 h3 + b4                                        W4: [3, 256]
With bf16=True the values the tensor-core kernel rounds to bfloat16 are
rounded here too (the features, the three hidden activations and W1's
feature part, W2, W3, W4); everything else stays FP64.
"""
from __future__ import annotations

import numpy as np

WIDTH = 256
NF = 64


def bf16(a):
    """Round to bfloat16 (nearest, ties to even) and back, via FP32."""
    x = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def features(x, Bf):
    """gamma(x) [N, 2 NF] of points x [N, 3]."""
    p = 2.0 * np.pi * (np.asarray(x, np.float64) @ np.asarray(Bf, np.float64).T)
    return np.concatenate([np.sin(p), np.cos(p)], axis=1)


def forward(x, theta, Bf, W1, b1, W2, b2, W3, b3, W4, b4, bf=False):
    """dx [N, 3] of points x [N, 3] at pose theta [P]."""
    r = bf16 if bf else (lambda a: np.asarray(a, np.float64))
    W1 = np.asarray(W1, np.float64)
    g = features(x, Bf)
    nf = g.shape[1]
    z1 = r(g) @ r(W1[:, :nf]).T + (W1[:, nf:] @ np.asarray(theta, np.float64) + np.asarray(b1, np.float64))
    h = np.maximum(z1, 0.0)
    for W, b in ((W2, b2), (W3, b3)):
        h = np.maximum(r(h) @ r(W).T + np.asarray(b, np.float64), 0.0)
    return r(h) @ r(W4).T + np.asarray(b4, np.float64)


__all__ = ["WIDTH", "NF", "bf16", "features", "forward"]
