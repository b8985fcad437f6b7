"""Oracle for the training-loop schedule of the appendix ("Experimental
Setup"): the position learning rate and the opacity reset.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU legs, never by the library's product path.

* Position learning rate: log-linear from 1.6e-4 at iteration 0 to 1.6e-6 at
  iteration 30,000 (the 3DGS convention the appendix keeps), held at the final
  value afterwards. The appendix's delay multiplier 0.01 acts only over a
  number of delay steps that it does not give (3DGS's default is 0), so it
  has no effect here (reading).
* Opacity reset every 3,000 iterations: every opacity above 0.01 is set to
  0.01 (logit = log(0.01 / 0.99)); the opacity group's Adam moments restart
  at zero.
"""
from __future__ import annotations

import math

import numpy as np

POS_LR_INIT = 1.6e-4
POS_LR_FINAL = 1.6e-6
POS_LR_STEPS = 30_000
RESET_EVERY = 3_000
RESET_OPACITY = 0.01


def position_lr(t: int, init: float = POS_LR_INIT, final: float = POS_LR_FINAL, steps: int = POS_LR_STEPS) -> float:
    s = min(max(t / steps, 0.0), 1.0)
    return math.exp((1.0 - s) * math.log(init) + s * math.log(final))


def opacity_reset(logits, m=None, v=None, max_opacity: float = RESET_OPACITY):
    """(logits, m, v) after the reset, FP64."""
    cap = math.log(max_opacity / (1.0 - max_opacity))
    lg = np.minimum(np.asarray(logits, np.float64), cap)
    z = lambda a: None if a is None else np.zeros_like(np.asarray(a, np.float64))
    return lg, z(m), z(v)
