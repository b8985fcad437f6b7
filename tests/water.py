"""Test-side composition of a synthetic underwater observation from the maps
drawn by ``scenes.water_view``: the per-pixel form of Eq. 5,
I = J exp(-beta_D z) + B_inf (1 - exp(-beta_B z)), with the direct signal J
removed in shadows and in open water (depth at z_far)."""
from __future__ import annotations

import numpy as np

from paper_2411_19588_b300 import scenes


def compose(depth, albedo, shadow, medium: scenes.Medium, z_far: float = 20.0) -> np.ndarray:
    z = np.asarray(depth, np.float64)
    J = np.asarray(albedo, np.float64) * (~np.asarray(shadow))[None]
    J[:, z >= z_far] = 0.0
    bd = np.asarray(medium.beta_d, np.float64)[:, None, None]
    bb = np.asarray(medium.beta_b, np.float64)[:, None, None]
    B = np.asarray(medium.b_inf, np.float64)[:, None, None]
    return (J * np.exp(-bd * z) + B * (1.0 - np.exp(-bb * z))).astype(np.float32)


def view(seed: int, width: int, height: int, **kw):
    """(image [3,H,W] f32, depth [H,W] f32, medium)."""
    depth, alb, shadow, med = scenes.water_view(seed, width, height, **kw)
    return compose(depth, alb, shadow, med), depth, med
