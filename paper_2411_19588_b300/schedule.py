"""The training schedule of the appendix ("Experimental Setup"): the
position learning rate decays log-linearly from 1.6e-4 to 1.6e-6 over
30,000 iterations (held at the final value after that), and every 3,000
iterations the opacities are reset to at most 0.01 (the 3DGS conventions the
paper keeps). Host-side scalars; the reset itself runs in libsplash
(render.opacity_reset); so do the densification statistics and step
(render.densify) on the schedule below."""
from __future__ import annotations

import math

POSITION_LR = (1.6e-4, 1.6e-6, 30_000)  # initial, final, steps
OPACITY_RESET_EVERY = 3_000
OPACITY_RESET_VALUE = 0.01
# densification: interval 100 from iteration 1,500 to 15,000, gradient threshold 0.0002,
# minimum opacity 0.1 (as printed), percent_dense 0.01 of the scene extent (3DGS)
DENSIFY = {"start": 1_500, "stop": 15_000, "every": 100, "grad_threshold": 0.0002, "min_opacity": 0.1,
           "percent_dense": 0.01}


def position_lr(it: int, init: float = POSITION_LR[0], final: float = POSITION_LR[1],
                steps: int = POSITION_LR[2]) -> float:
    """Learning rate of the Gaussian centres at iteration `it` (0-based)."""
    frac = min(1.0, max(0.0, it / steps))
    return math.exp(math.log(init) * (1.0 - frac) + math.log(final) * frac)
