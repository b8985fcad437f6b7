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


def _decisions(log_scales, opacity_logits, stats, threshold, min_opacity, dense):
    """The three decisions of every Gaussian, each taken in FP64 on its
    definition, with its relative distance to the threshold:
    low opacity sigmoid(o) < min_opacity, selection mean gradient >=
    threshold, size max(exp(s)) > dense."""
    ls = np.asarray(log_scales, np.float64)
    lg = np.asarray(opacity_logits, np.float64)
    st = np.asarray(stats, np.float64).reshape(-1, 2)
    opac = 1.0 / (1.0 + np.exp(-lg))
    avg = st[:, 0] / np.maximum(st[:, 1], 1.0)
    size = np.exp(ls.max(axis=1)) if len(ls) else np.zeros(0)
    take = np.stack([opac < min_opacity, avg >= threshold, size > dense], 1)
    dist = np.stack([np.abs(opac - min_opacity) / min_opacity, np.abs(avg - threshold) / threshold,
                     np.abs(size - dense) / dense], 1)
    return take, dist


LOW_OPACITY, SELECTED, LARGE = 1, 2, 4


def decision_margins(log_scales, opacity_logits, stats, threshold=THRESHOLD, min_opacity=MIN_OPACITY, dense=1.0):
    """[n, 3] relative distances of the low-opacity, selection and size
    decisions to their thresholds (bits LOW_OPACITY, SELECTED, LARGE of a flip
    mask, in that order)."""
    return _decisions(log_scales, opacity_logits, stats, threshold, min_opacity, dense)[1]


def classify(log_scales, opacity_logits, stats, threshold=THRESHOLD, min_opacity=MIN_OPACITY, dense=1.0, flip=None):
    """Action per Gaussian from the three FP64 decisions. ``flip`` (optional,
    one bit mask per Gaussian of LOW_OPACITY | SELECTED | LARGE) takes the
    named decisions the other way: where a decision lies within rounding of
    its threshold an FP32 evaluation may take either outcome."""
    take, _ = _decisions(log_scales, opacity_logits, stats, threshold, min_opacity, dense)
    if flip is not None:
        f = np.asarray(flip, np.int64).reshape(-1)
        take = take ^ np.stack([(f & LOW_OPACITY) > 0, (f & SELECTED) > 0, (f & LARGE) > 0], 1)
    low, sel, big = take[:, 0], take[:, 1], take[:, 2]
    act = np.full(len(take), KEEP, np.int64)
    act[sel & ~big] = CLONE
    act[sel & big] = SPLIT
    act[low] = PRUNE
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
