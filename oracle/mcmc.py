"""Oracle for the MCMC densification the paper adopts, FP64 numpy.

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the
benchmark's CPU legs, never by the library's product path.

Sec. IV-D replaces the 3DGS densification (clone / split / prune) by the
sampling form of 3DGS-MCMC, and Sec. VI ablates that choice. The paper
gives no formulas of its own; this states the cited method's relocation
and position noise as the build reads them (the readings are listed in the
design notes):

Relocation (the densification interval of the schedule):
  * dead: sigmoid(o) <= min_opacity (0.005), decided in FP64;
  * every dead Gaussian d draws a source among the live ones with
    probability proportional to opacity: with C the inclusive running sum of
    the weights w_g = sigmoid(o_g) for live g, 0 for dead g, in index order,
    and u_d in [0, 1) given, the source is the first g with
    C_g > u_d C_total;
  * a source g drawn c_g times stands for N = min(c_g + 1, 51) Gaussians (g
    and its c_g copies). All of them take opacity
        o' = 1 - (1 - o)^(1/N)
    (N copies composited at one point give the old opacity back) and scales
        s' = s * o / Z,  Z = sum_{i=1}^{N} sum_{k=0}^{i-1} C(i-1, k) (-1)^k o'^(k+1) / sqrt(k+1)
    (the integral of the composite 1 - (1 - o' e^{-x^2/2s'^2})^N along a
    line equals that of o e^{-x^2/2s^2});
  * a copy takes every other parameter of its source; the Adam moments of
    the sources and of the copies start at zero.

Position noise (every iteration, after the Adam step):
    mu <- mu + lambda_noise * lr_mu * sigmoid(-k (o - t)) * Sigma eta,
  Sigma = R diag(s)^2 R^T the Gaussian's covariance, eta ~ N(0, I) given,
  k = 100, t = 0.005.
"""
from __future__ import annotations

import math

import numpy as np

MIN_OPACITY = 0.005
N_MAX = 51
NOISE_K = 100.0
NOISE_T = 0.005
LAMBDA_NOISE = 5e5


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def dead_margins(opacity_logits, min_opacity=MIN_OPACITY):
    """Relative distance of each opacity to the dead threshold."""
    o = _sigmoid(opacity_logits)
    return np.abs(o - min_opacity) / min_opacity


def sources(opacity_logits, uniforms, min_opacity=MIN_OPACITY, dead_flip=None):
    """(dead mask, source index per Gaussian (-1 where live)). dead_flip
    (optional bool mask) takes the dead / live decision the other way."""
    o = _sigmoid(opacity_logits)
    dead = o <= min_opacity
    if dead_flip is not None:
        dead = dead ^ np.asarray(dead_flip, bool)
    w = np.where(dead, 0.0, o)
    C = np.cumsum(w)
    src = np.full(len(o), -1, np.int64)
    if len(o) == 0 or C[-1] <= 0.0:
        return dead, src
    u = np.asarray(uniforms, np.float64)
    for d in np.flatnonzero(dead):
        src[d] = int(np.searchsorted(C, u[d] * C[-1], side="right"))
    return dead, src


def z_factor(N: int, o_new: float) -> float:
    """Z = sum_{i=1}^{N} sum_{k=0}^{i-1} C(i-1, k) (-1)^k o'^(k+1) / sqrt(k+1)."""
    z = 0.0
    for i in range(1, N + 1):
        for k in range(i):
            z += math.comb(i - 1, k) * (-1) ** k * o_new ** (k + 1) / math.sqrt(k + 1)
    return z


def shared_opacity_scale(o: float, N: int):
    """(o', scale factor s'/s) of a source standing for N Gaussians."""
    o_new = 1.0 - (1.0 - o) ** (1.0 / N)
    return o_new, o / z_factor(N, o_new)


def relocate(params: dict, m: dict, v: dict, uniforms, min_opacity=MIN_OPACITY, dead_flip=None):
    """New (params, m, v) dicts (FP64) after one relocation, and the number of
    dead Gaussians. Keys: means, log_scales, quats, opacity_logits, sh."""
    P = {k: np.array(params[k], np.float64) for k in params}
    M = {k: np.array(m[k], np.float64) for k in m}
    V = {k: np.array(v[k], np.float64) for k in v}
    dead, src = sources(P["opacity_logits"], uniforms, min_opacity, dead_flip)
    n_dead = int(dead.sum())
    if n_dead == 0 or (src[dead] < 0).any():
        return P, M, V, n_dead
    counts = np.bincount(src[dead], minlength=len(dead))
    for g in np.flatnonzero(counts):
        N = min(int(counts[g]) + 1, N_MAX)
        o = float(_sigmoid(P["opacity_logits"][g]))
        o_new, f = shared_opacity_scale(o, N)
        P["opacity_logits"][g] = math.log(o_new / (1.0 - o_new))
        P["log_scales"][g] = P["log_scales"][g] + math.log(f)
        for k in M:
            M[k][g] = 0.0
            V[k][g] = 0.0
    for d in np.flatnonzero(dead):
        g = src[d]
        for k in P:
            P[k][d] = P[k][g]
        for k in M:
            M[k][d] = 0.0
            V[k][d] = 0.0
    return P, M, V, n_dead


def rotation(q) -> np.ndarray:
    """Rotation matrix of a (w, x, y, z) quaternion after normalisation."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def noise(means, log_scales, quats, opacity_logits, eta, lr: float, lambda_noise=LAMBDA_NOISE):
    """Means after the position noise (FP64)."""
    mu = np.array(means, np.float64)
    o = _sigmoid(opacity_logits)
    gate = 1.0 / (1.0 + np.exp(NOISE_K * (o - NOISE_T)))  # sigmoid(-k (o - t))
    for i in range(len(mu)):
        R = rotation(quats[i])
        s2 = np.exp(2.0 * np.asarray(log_scales[i], np.float64))
        Sigma = R @ np.diag(s2) @ R.T
        mu[i] += lambda_noise * lr * gate[i] * (Sigma @ np.asarray(eta[i], np.float64))
    return mu
