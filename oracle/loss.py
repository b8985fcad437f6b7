"""Image loss oracle: L1 + lam * (1 - SSIM), FP64, plain PyTorch CPU ops.

TEST INFRASTRUCTURE ONLY. The paper's photometric term is Eq. 7
(1 - lambda) L1 + lambda D-SSIM over the rendered and observed images; the
training-step workload uses L1 + 0.2 (1 - SSIM). SSIM follows the usual
definition (Wang et al.) that 3DGS uses: an 11x11 Gaussian window with
sigma = 1.5 normalised to sum 1, per-channel local statistics with zero
padding of 5, C1 = 0.01^2, C2 = 0.03^2, mean over channels and pixels.
Gradients come from autograd (a library primitive) on this definition.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window() -> torch.Tensor:
    x = torch.arange(WINDOW, dtype=torch.float64) - (WINDOW // 2)
    g = torch.exp(-(x ** 2) / (2 * SIGMA ** 2))
    g = g / g.sum()
    return torch.outer(g, g)


def _blur(x: torch.Tensor) -> torch.Tensor:
    """Per-channel 2D correlation of (C, H, W) with the window, zero padding."""
    C = x.shape[0]
    w = window().expand(C, 1, WINDOW, WINDOW).contiguous()
    return F.conv2d(x[None], w, padding=WINDOW // 2, groups=C)[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    mx, my = _blur(x), _blur(y)
    sxx = _blur(x * x) - mx * mx
    syy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(x, y) -> float:
    x = torch.as_tensor(np.asarray(x, np.float64))
    y = torch.as_tensor(np.asarray(y, np.float64))
    return float(ssim_map(x, y).mean())


def loss_and_grad(img, target, lam: float = 0.2):
    """Returns (loss, dloss/dimg) for loss = mean|img - target| + lam (1 - mean SSIM)."""
    x = torch.tensor(np.asarray(img, np.float64), requires_grad=True)
    y = torch.as_tensor(np.asarray(target, np.float64))
    loss = (x - y).abs().mean() + lam * (1 - ssim_map(x, y).mean())
    loss.backward()
    return float(loss), x.grad.numpy().copy()
