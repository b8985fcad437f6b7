"""Pins of the training-loop schedule oracle (appendix, "Experimental Setup")."""
import math

import numpy as np

from oracle import schedule as S


def test_position_lr_end_points_midpoint_and_clamp():
    assert S.position_lr(0) == 1.6e-4
    assert math.isclose(S.position_lr(30_000), 1.6e-6, rel_tol=1e-12)
    assert math.isclose(S.position_lr(15_000), math.sqrt(1.6e-4 * 1.6e-6), rel_tol=1e-12)  # geometric mean
    assert S.position_lr(45_000) == S.position_lr(30_000)
    lrs = [S.position_lr(t) for t in range(0, 30_001, 1000)]
    assert all(a > b for a, b in zip(lrs, lrs[1:]))
    # a constant ratio per step: log-linear
    r = [lrs[i + 1] / lrs[i] for i in range(len(lrs) - 1)]
    assert max(r) - min(r) < 1e-12


def test_opacity_reset_caps_at_one_percent_and_clears_moments():
    logits = np.array([-8.0, -4.6, -4.5, 0.0, 3.0])
    lg, m, v = S.opacity_reset(logits, np.ones(5), np.ones(5))
    p = 1 / (1 + np.exp(-lg))
    assert np.all(p <= 0.01 + 1e-15)
    assert lg[0] == -8.0 and lg[1] == -4.6          # already below 1 %: untouched
    assert np.allclose(p[2:], 0.01)
    assert np.all(m == 0) and np.all(v == 0)
