"""Oracle for water removal from a rendered depth map (the application of
Sec. I and Sec. V: "clean" colour from the reconstructed depth and water),
FP64 numpy.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU legs, never by the library's product path.

The per-pixel image formation of Eq. 5, I = J a + B_inf (1 - b) with
a = exp(-beta_D z) and b = exp(-beta_B z), is inverted for J at every pixel
given the depth z (Eq. 6's expected depth) and the water medium
(beta_D[3], beta_B[3], B_inf[3]):

    J = max(I - B_inf (1 - b), 0) / a

The direct signal I - B_inf (1 - b) is physical only where non-negative
(reading: a pixel darker than the modelled backscatter has no direct light
left), so it is clipped at 0 before the attenuation is undone.

The clean render (water removed) of a scene is the renderer with the medium
set to zero: Eq. 5 with beta_D = beta_B = B_inf = 0 is the plain composite of
Eq. 1, which the rasterizer's oracle already pins.
"""
from __future__ import annotations

import numpy as np


def restore(image, depth, medium) -> np.ndarray:
    """J [3,H,W] from an observed image [3,H,W], depth [H,W] and medium [9]."""
    img = np.asarray(image, np.float64)
    z = np.asarray(depth, np.float64)[None]
    med = np.asarray(medium, np.float64)
    bD, bB, B = (med[0:3, None, None], med[3:6, None, None], med[6:9, None, None])
    direct = np.maximum(img - B * (1.0 - np.exp(-bB * z)), 0.0)
    return direct * np.exp(bD * z)
