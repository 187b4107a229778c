"""FP64 oracle of the Adam update that trains the avatar's parameters
(Kingma and Ba's algorithm, the optimiser of the 3DGS training the paper
builds on; Sec. 3.3 and Sec. 4 give the losses and schedules, not the
update).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

Step t (1-based) of one parameter group with learning rate lr:
  m <- b1 m + (1 - b1) g
  v <- b2 v + (1 - b2) g^2
  p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
With bf16=True the parameter is stored as bfloat16: the update is computed
from its stored value and the result rounded to bfloat16 (nearest, ties to
even); m and v stay FP64 here (FP32 in the kernel).
"""
from __future__ import annotations

import numpy as np

from .mlp import bf16 as _bf16


def step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-15, bf16=False):
    """One Adam step; returns (p, m, v) as new FP64 arrays."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    p = p - lr * mh / (np.sqrt(vh) + eps)
    if bf16:
        p = _bf16(p)
    return p, m, v


__all__ = ["step"]
