"""Adam oracle, FP64 numpy, textbook form (Kingma & Ba, Algorithm 1).

TEST INFRASTRUCTURE ONLY. Sec. IV-C optimises all Gaussian and medium
parameters with Adam at the 3DGS learning rates (appendix "Experimental
Setup"). Bias-corrected step:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
optionally followed by a lower clamp of the parameter.
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15,
              clamp_min=None):
    p = np.asarray(p, np.float64).copy()
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    if clamp_min is not None:
        p = np.maximum(p, clamp_min)
    return p, m, v
