"""Oracle for the densification step of the training loop (appendix,
"Experimental Setup": densification interval 100 from iteration 1,500 to
15,000, gradient threshold 0.0002, minimum opacity 0.1; the 3DGS procedure
the paper keeps), FP64 numpy.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU legs, never by the library's product path.

Statistics, every iteration, for every Gaussian in the view (not culled):
    accum += || (g_x W / 2, g_y H / 2) ||,  count += 1,
with (g_x, g_y) the loss gradient w.r.t. the Gaussian's projected centre in
pixels (so the norm is taken in normalised device coordinates, as 3DGS does).

Densification step, per Gaussian (avg = accum / max(count, 1)):
    prune  if sigmoid(opacity logit) < min_opacity       -> no output
    split  elif avg >= threshold and max scale > dense   -> two new Gaussians
    clone  elif avg >= threshold                         -> itself and a copy
    keep   otherwise                                     -> itself
with dense = percent_dense (0.01) x scene extent. Outputs follow the input
order (a Gaussian's outputs are consecutive). A split Gaussian is replaced by
two samples mu + R diag(s) eps_k (eps_k the k-th of two given standard normal
3-vectors, R the rotation of the normalised quaternion, s = exp(log-scales)),
with log-scales lowered by log(1.6) and every other parameter copied. The
Adam moments of kept Gaussians and of a clone's original carry over; a
clone's copy and split samples start at zero.

Readings: the paper cites 3DGS-MCMC for densification but lists 3DGS's
clone/split/prune hyper-parameters; the listed procedure is followed, with
its minimum opacity 0.1 as printed. 3DGS's additional pruning of very large
Gaussians (screen or world size) is not in the paper and not applied.
"""
from __future__ import annotations

import math

import numpy as np

THRESHOLD = 0.0002
MIN_OPACITY = 0.1
PERCENT_DENSE = 0.01
SPLIT_SCALE = 1.6
PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3


def stat_increment(g_proj_xy, width: int, height: int) -> np.ndarray:
    """Per-Gaussian NDC gradient norm from pixel-space centre gradients [n, 2]."""
    g = np.asarray(g_proj_xy, np.float64)
    return np.hypot(g[:, 0] * width / 2.0, g[:, 1] * height / 2.0)


def classify(log_scales, opacity_logits, stats, threshold=THRESHOLD, min_opacity=MIN_OPACITY, dense=1.0):
    """Action per Gaussian. The three integer decisions are taken in FP32
    on the stored values (the kernel's precision): opacity below
    min_opacity as logit < fl32(logit(min_opacity)), size as max log-scale >
    fl32(log(dense)), selection as fl32(accum / max(count, 1)) >= fl32(threshold)."""
    ls = np.asarray(log_scales, np.float32)
    lg = np.asarray(opacity_logits, np.float32)
    st = np.asarray(stats, np.float32)
    avg = st[:, 0] / np.maximum(st[:, 1], np.float32(1.0))
    big = ls.max(axis=1) > np.float32(math.log(dense))
    sel = avg >= np.float32(threshold)
    act = np.full(len(lg), KEEP, np.int64)
    act[sel & ~big] = CLONE
    act[sel & big] = SPLIT
    act[lg < np.float32(math.log(min_opacity / (1.0 - min_opacity)))] = PRUNE
    return act


def rotation(q) -> np.ndarray:
    """Rotation matrix of a (w, x, y, z) quaternion after normalisation."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def apply(params: dict, m: dict, v: dict, actions, noise):
    """New (params, m, v) dicts (keys means, log_scales, quats, opacity_logits,
    sh) after the step; noise [n, 2, 3] standard normals (used by splits)."""
    out_p = {k: [] for k in params}
    out_m = {k: [] for k in params}
    out_v = {k: [] for k in params}
    noise = np.asarray(noise, np.float64)

    def emit(i, src, moments):
        for k in params:
            out_p[k].append(np.asarray(src[k], np.float64))
            zero = np.zeros_like(np.asarray(params[k][i], np.float64))
            out_m[k].append(np.asarray(m[k][i], np.float64) if moments else zero)
            out_v[k].append(np.asarray(v[k][i], np.float64) if moments else zero)

    for i, a in enumerate(np.asarray(actions)):
        one = {k: np.asarray(params[k][i], np.float64) for k in params}
        if a == KEEP:
            emit(i, one, True)
        elif a == CLONE:
            emit(i, one, True)
            emit(i, one, False)
        elif a == SPLIT:
            R = rotation(one["quats"])
            s = np.exp(one["log_scales"])
            for k in range(2):
                new = dict(one)
                new["means"] = one["means"] + R @ (s * noise[i, k])
                new["log_scales"] = one["log_scales"] - math.log(SPLIT_SCALE)
                emit(i, new, False)
    shape = lambda k: (0,) + np.asarray(params[k]).shape[1:]
    stack = lambda d: {k: (np.stack(d[k]) if d[k] else np.zeros(shape(k))) for k in d}
    return stack(out_p), stack(out_m), stack(out_v)
