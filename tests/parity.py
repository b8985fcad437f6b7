"""Helpers shared by the GPU parity tests: run the CUDA path through the
C ABI (via the package binding) and the FP64 oracle on the same seeded
inputs, and compare them with the protocol below.

Comparison protocol:
  * a decision of the method (a Gaussian's 3-sigma cut at a pixel, the
    alpha < 1/255 skip, the transmittance stop, and the order of two
    Gaussians whose depths are equal at FP32 resolution) whose FP64 quantity
    lies within oracle.NEAR (relative) of its threshold may be taken either
    way by an FP32 evaluation of the same definition. The oracle lists such
    near decisions per pixel and renders the pixel under every combination
    of their outcomes (its branches, up to 4 near decisions); a pixel
    passes when the GPU matches one branch in every output (image, depth,
    logistic depth) at the tolerances below. Every other pixel has one
    branch, the FP64 walk;
  * pixels with more near decisions than the oracle enumerates are excluded
    and counted: at most MAX_EXCLUDED of the pixels (0.1 %);
  * image and logistic depth: |gpu - oracle| <= 1e-5; metric depth:
    |gpu - oracle| <= 1e-5 * oracle;
  * gradients: the oracle's adjoint is taken on the branch the GPU's
    forward matched. Upstream gradients are zeroed (on both sides, counted)
    at excluded pixels, at pixels that two branches match (the forward
    cannot tell which the GPU took) and at pixels whose contributors lie
    within GMARGIN of a gradient kink (the alpha clamp at 0.99, the colour
    clamp at 0, the Jacobian clamp); then every component obeys
    |gpu - oracle| <= 1e-3 |oracle| + GRAD_FLOOR * max|oracle| of its array.

Each comparison appends its counts to PARITY_LOG; the test session prints
them in its summary.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

MARGIN = oracle.NEAR
GMARGIN = 1e-4
MAX_EXCLUDED = 1e-3
IMG_ATOL = 1e-5
DEPTH_RTOL = 1e-5
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-5
NEAR_MAX = 4

PARITY_LOG: list = []


def medium_tensor(medium) -> torch.Tensor:
    return torch.tensor(medium.as_array(), dtype=torch.float32, device="cuda")


def gpu_forward(renderer, g, medium, cam, state=None):
    params = R.params_to_device(g)
    med = medium_tensor(medium)
    st = state or renderer.state()
    img, depth, depth01 = renderer.forward(st, params, med, cam)
    torch.cuda.synchronize()
    return {"image": img.cpu().numpy().astype(np.float64), "depth": depth.cpu().numpy().astype(np.float64),
            "depth01": depth01.cpu().numpy().astype(np.float64), "state": st, "params": params, "medium": med}


def _errors(gi, gd, g01, img, dep, d01):
    """Per-pixel worst error of the three outputs in units of its tolerance
    (<= 1 passes). gi, img: (3, ...); the rest shaped like one channel."""
    e_img = np.abs(gi - img).max(axis=0) / IMG_ATOL
    e_dep = np.abs(gd - dep) / (DEPTH_RTOL * np.maximum(dep, 1e-30))
    e_01 = np.abs(g01 - d01) / IMG_ATOL
    return np.maximum(np.maximum(e_img, e_dep), e_01)


def compare_forward(gpu, ora, pix=None, label="", scene=None, max_excluded=MAX_EXCLUDED,
                    branches=oracle.branches):
    """gpu: full-image arrays; ora: oracle render over all pixels (pix=None)
    or over the listed linear pixel indices; scene = (g, medium, cam) lets
    the oracle render the branches of pixels with near decisions (without
    it those pixels are excluded and counted); ``branches`` renders them
    (the segment form's oracle by default).

    Returns the error statistics and, shaped like the oracle's arrays,
    ``branch`` (the branch each pixel matched), ``excluded`` and ``multi``
    (more than one branch matched)."""
    if pix is None:
        gi, gd, g01 = gpu["image"], gpu["depth"], gpu["depth01"]
        lin = np.arange(gi.shape[1] * gi.shape[2])
    else:
        W = gpu["image"].shape[2]
        lin = np.asarray(pix).reshape(-1)
        iy, ix = np.divmod(lin, W)
        gi, gd, g01 = gpu["image"][:, iy, ix], gpu["depth"][iy, ix], gpu["depth01"][iy, ix]
    shape = ora["depth"].shape
    n = int(np.prod(shape))
    gi, gd, g01 = gi.reshape(3, n), gd.reshape(n), g01.reshape(n)
    n_near = ora["n_near"].reshape(n)
    img, dep, d01 = ora["image"].reshape(3, n).copy(), ora["depth"].reshape(n).copy(), ora["depth01"].reshape(n).copy()
    branch = np.zeros(n, np.int64)
    multi = np.zeros(n, bool)
    excluded = n_near > NEAR_MAX
    amb = np.flatnonzero((n_near > 0) & ~excluded)
    if scene is None:
        excluded[amb] = True
    elif amb.size:
        g, m, cam = scene
        br = branches(g, m, cam, lin[amb])
        e = _errors(gi[:, amb, None], gd[amb, None], g01[amb, None], br["image"], br["depth"], br["depth01"])
        e = np.where(br["valid"], e, np.inf)
        best = e.argmin(axis=1)
        rows = np.arange(amb.size)
        branch[amb] = best
        multi[amb] = (e <= 1.0).sum(axis=1) > 1
        img[:, amb] = br["image"][:, rows, best]
        dep[amb] = br["depth"][rows, best]
        d01[amb] = br["depth01"][rows, best]
    ok = ~excluded
    err = _errors(gi, gd, g01, img, dep, d01)
    frac = float(excluded.mean()) if n else 0.0
    stats = {"label": label, "pixels": n, "near": int((n_near > 0).sum()), "alt_branch": int((branch > 0).sum()),
             "multi": int(multi.sum()), "excluded": int(excluded.sum()), "excluded_frac": frac,
             "img_max": float(np.abs(gi - img)[:, ok].max(initial=0)),
             "depth_rel_max": float((np.abs(gd - dep) / np.maximum(dep, 1e-30))[ok].max(initial=0)),
             "depth01_max": float(np.abs(g01 - d01)[ok].max(initial=0))}
    PARITY_LOG.append(stats)
    assert frac <= max_excluded, f"{label}: {excluded.sum()} excluded pixels ({frac:.2e})"
    bad = np.flatnonzero(ok & (err > 1.0))
    assert bad.size == 0, (label, f"{bad.size} pixels match no branch", bad[:5], err[bad[:5]], n_near[bad[:5]], stats)
    return dict(stats, branch=branch.reshape(shape), excluded=excluded.reshape(shape), multi=multi.reshape(shape))


def upstream_keep(ora, fwd):
    """Pixels whose upstream gradient stays non-zero: resolved to exactly one
    branch and clear of gradient kinks. Counted into the last PARITY_LOG
    entry of the forward comparison ``fwd``."""
    keep = ~fwd["excluded"] & ~fwd["multi"] & (ora["gmargin"] >= GMARGIN)
    for s in reversed(PARITY_LOG):
        if s["label"] == fwd["label"]:
            s["grad_zeroed"] = int(keep.size - keep.sum())
            break
    return keep


def compare_grads(gpu: dict, ora: dict, label=""):
    worst = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "medium"):
        a = np.asarray(gpu[k], np.float64).reshape(-1)
        b = np.asarray(ora[k], np.float64).reshape(-1)
        scale = np.abs(b).max(initial=0.0)
        tol = GRAD_RTOL * np.abs(b) + GRAD_FLOOR * scale
        err = np.abs(a - b)
        viol = err > tol
        worst[k] = float((err / np.maximum(tol, 1e-300)).max(initial=0.0))
        assert not viol.any(), (label, k, int(viol.sum()), a[viol][:5], b[viol][:5])
    return worst


def grads_to_numpy(grads: dict) -> dict:
    return {k: v.detach().cpu().numpy() for k, v in grads.items()}
