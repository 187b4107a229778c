"""FP64 oracle of the image loss of Eq. 5 (Sec. 3.3): the 3DGS loss
L_img = (1 - lambda) L1 + lambda D-SSIM, D-SSIM = 1 - SSIM.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.

SSIM follows its definition (structural similarity of Wang et al.): per
channel and pixel, local means, variances and covariance under an 11 x 11
Gaussian window (sigma 1.5, normalised) with zero padding at the image border
(the 3DGS convention), C1 = 0.01^2, C2 = 0.03^2,
  SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
averaged over channels and pixels.  The windowed means are a library
convolution (scipy.ndimage); the gradient is FP64 autograd through
torch.nn.functional.conv2d.
"""
from __future__ import annotations

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gauss_1d(n=WIN, sigma=SIGMA):
    x = np.arange(n) - (n - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(a):
    """Windowed mean of a [C, H, W] array, zero padding."""
    from scipy import ndimage
    w = np.outer(gauss_1d(), gauss_1d())
    return np.stack([ndimage.convolve(a[c], w, mode="constant", cval=0.0) for c in range(a.shape[0])])


def ssim_map(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def image_loss(img, target, lam=0.2):
    """(1 - lam) mean |img - target| + lam (1 - mean SSIM); img, target [C, H, W]."""
    img = np.asarray(img, np.float64)
    target = np.asarray(target, np.float64)
    l1 = np.abs(img - target).mean()
    return (1.0 - lam) * l1 + lam * (1.0 - ssim_map(img, target).mean())


def image_loss_torch(x, y, lam=0.2):
    """The same definition on FP64 torch tensors [C, H, W] (differentiable)."""
    import torch
    import torch.nn.functional as F
    C = x.shape[0]
    g = torch.tensor(gauss_1d(), dtype=torch.float64)
    w = torch.outer(g, g).expand(C, 1, WIN, WIN).contiguous()

    def blur(a):
        return F.conv2d(a[None], w, padding=WIN // 2, groups=C)[0]

    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    s = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return (1.0 - lam) * (x - y).abs().mean() + lam * (1.0 - s.mean())


def image_loss_grad(img, target, lam=0.2):
    """(loss, dloss/dimg) by FP64 autograd of the same definition."""
    import torch
    x = torch.tensor(np.asarray(img, np.float64), requires_grad=True)
    y = torch.tensor(np.asarray(target, np.float64))
    loss = image_loss_torch(x, y, lam)
    loss.backward()
    return float(loss.detach()), x.grad.numpy()


__all__ = ["gauss_1d", "ssim_map", "image_loss", "image_loss_torch", "image_loss_grad", "WIN", "SIGMA", "C1",
           "C2"]
