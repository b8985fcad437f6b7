"""FP64 CPU oracle for the Gaussian Splashing rasterizer.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct statement of
what the CUDA path computes. Only ``tests/``, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` / reference legs may import it. It shares no
code with the package ``paper_2411_19588_b300``; both are fed from the seeded
generators in ``paper_2411_19588_b300.scenes``, which hold no rendering
arithmetic.

Contents:
  * ``splash_oracle.c`` (via ctypes): projection, per-pixel compositing with
    the water model over the full depth-sorted list (no tiling), and the
    analytic FP64 adjoint. Passages: Eq. 1-6, Sec. III-A, Sec. IV-A/B/D.
  * ``loss``: L1 + lambda (1 - SSIM) with autograd in FP64 (Eq. 7 form).
  * ``adam``: one Adam step, textbook form (Sec. IV-C uses Adam).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_NPROJ = _NPIX = _NGP = None

PROJ_FIELDS = ["vis", "x", "y", "KA", "KB", "KC", "SA", "SB", "SC", "opac", "col_r", "col_g", "col_b",
               "a_r", "a_g", "a_b", "b_r", "b_g", "b_b", "d", "raw_r", "raw_g", "raw_b", "cull_margin",
               "tx", "ty", "gmargin"]
PIX_FIELDS = ["r", "g", "b", "depth", "depth01", "T_f", "n_contrib", "acc", "margin", "gmargin", "tie",
              "n_cand", "dsum", "n_iter", "n_near"]
BRANCH_FIELDS = ["r", "g", "b", "depth", "depth01", "T_f", "n_contrib", "valid"]
# A decision (3-sigma cut, alpha skip, transmittance stop, FP32 depth order)
# whose FP64 quantity lies within NEAR (relative) of its threshold may be
# taken either way by an FP32 evaluation of the same definition.
NEAR = 1e-5


def lib():
    global _lib, _NPROJ, _NPIX, _NGP
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        i64, ci, cd = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.oracle_project.argtypes = [i64, dp, dp, dp, dp, dp, ci, dp, dp, dp, ci]
        L.oracle_render.argtypes = [i64, dp, dp, dp, dp, dp, ci, dp, dp, i64, ip, cd, ci, dp, ci]
        L.oracle_render_branches.argtypes = [i64, dp, dp, dp, dp, dp, ci, dp, dp, i64, ip, cd, ci, dp, ci]
        L.oracle_backward.argtypes = [i64, dp, dp, dp, dp, dp, ci, dp, dp, i64, ip, dp, ip, cd, ci,
                                      dp, dp, dp, dp, dp, dp, dp, ci]
        L.oracle_composite.argtypes = [i64, dp, dp, dp, dp, cd, dp]
        L.oracle_sh_basis.argtypes = [ci, dp, dp]
        for f in (L.oracle_project, L.oracle_render, L.oracle_render_branches, L.oracle_backward,
                  L.oracle_composite, L.oracle_sh_basis):
            f.restype = ci
        _NPROJ, _NPIX, _NGP = L.oracle_nproj(), L.oracle_npix(), L.oracle_ngproj()
        assert _NPROJ == len(PROJ_FIELDS) and _NPIX == len(PIX_FIELDS)
        assert L.oracle_nbf() == len(BRANCH_FIELDS)
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _params(g, medium, cam):
    arrs = [_d(x) for x in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
    med = _d(np.asarray(medium.as_array() if hasattr(medium, "as_array") else medium, np.float64))
    c = _d(cam.as_array() if hasattr(cam, "as_array") else cam)
    return arrs, med, c


def project(g, medium, cam, nthreads: int = 0) -> dict:
    """Per-Gaussian projection in FP64 (fields ``PROJ_FIELDS``)."""
    L = lib()
    arrs, med, c = _params(g, medium, cam)
    out = np.zeros((g.n, _NPROJ), np.float64)
    rc = L.oracle_project(g.n, *[p for _, p in arrs], g.sh_degree, med[1], c[1],
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_project failed: {rc}")
    return {k: out[:, i] for i, k in enumerate(PROJ_FIELDS)}


def _pix(cam, pix):
    if pix is None:
        return int(cam.width * cam.height), None, None
    p = np.ascontiguousarray(pix, dtype=np.int64)
    return int(p.size), p, p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def render(g, medium, cam, pix=None, nthreads: int = 0, near: float = NEAR, bin: int = 0) -> dict:
    """Render every pixel (``pix=None``; arrays shaped (H, W), image (3, H, W))
    or the listed linear pixel indices (arrays shaped (npix,), image (3, npix)).
    ``n_near`` counts each pixel's decisions within ``near`` of a threshold.
    ``bin`` > 0 scans, per pixel, only the Gaussians whose widened 3-sigma box
    meets its bin x bin block (same results, much faster on large scenes)."""
    L = lib()
    arrs, med, c = _params(g, medium, cam)
    npix, p, pp = _pix(cam, pix)
    out = np.zeros((npix, _NPIX), np.float64)
    rc = L.oracle_render(g.n, *[q for _, q in arrs], g.sh_degree, med[1], c[1], npix, pp, float(near), int(bin),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_render failed: {rc}")
    shape = (cam.height, cam.width) if pix is None else (npix,)
    res = {k: out[:, i].reshape(shape) for i, k in enumerate(PIX_FIELDS)}
    res["image"] = np.stack([res["r"], res["g"], res["b"]])
    return res


def branches(g, medium, cam, pix, nthreads: int = 0, near: float = NEAR, bin: int = 0) -> dict:
    """Every branch of the listed linear pixel indices: each field shaped
    (npix, NBRANCH). Branch b takes near decision i (in the FP64 walk's order)
    the other way when bit i of b is set; branch 0 is ``render``'s result.
    ``valid`` marks the 2^k branches of a pixel with k <= log2(NBRANCH) near
    decisions (branch 0 alone when it has more)."""
    L = lib()
    arrs, med, c = _params(g, medium, cam)
    p = np.ascontiguousarray(pix, dtype=np.int64).reshape(-1)
    nb = L.oracle_nbranch()
    out = np.zeros((p.size, nb, len(BRANCH_FIELDS)), np.float64)
    rc = L.oracle_render_branches(g.n, *[q for _, q in arrs], g.sh_degree, med[1], c[1], p.size,
                                  p.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), float(near), int(bin),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_render_branches failed: {rc}")
    res = {k: out[:, :, i] for i, k in enumerate(BRANCH_FIELDS)}
    res["image"] = np.stack([res["r"], res["g"], res["b"]])
    res["valid"] = res["valid"] > 0
    return res


def backward(g, medium, cam, dL_dimage, dL_ddepth=None, dL_ddepth01=None, pix=None, nthreads: int = 0,
             branch=None, near: float = NEAR, bin: int = 0) -> dict:
    """Gradients of L = <dL_dimage, C> + <dL_ddepth, z> + <dL_ddepth01, z01>
    with respect to every parameter (FP64 analytic adjoint). Upstream arrays
    are (3, H, W)/(H, W) for ``pix=None`` or (3, npix)/(npix,) otherwise.
    ``branch`` (optional, one int per pixel, shaped like a depth map) picks the
    branch of each pixel's near decisions whose adjoint is taken (see
    ``branches``); 0 everywhere is the FP64 walk."""
    L = lib()
    arrs, med, c = _params(g, medium, cam)
    npix, p, pp = _pix(cam, pix)
    gout = np.zeros((npix, 5), np.float64)
    gout[:, 0:3] = np.asarray(dL_dimage, np.float64).reshape(3, npix).T
    if dL_ddepth is not None:
        gout[:, 3] = np.asarray(dL_ddepth, np.float64).reshape(npix)
    if dL_ddepth01 is not None:
        gout[:, 4] = np.asarray(dL_ddepth01, np.float64).reshape(npix)
    K = (g.sh_degree + 1) ** 2
    res = {"means": np.zeros((g.n, 3)), "log_scales": np.zeros((g.n, 3)), "quats": np.zeros((g.n, 4)),
           "opacity_logits": np.zeros(g.n), "sh": np.zeros((g.n, K, 3)), "medium": np.zeros(9),
           "proj": np.zeros((g.n, _NGP))}
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    br = None if branch is None else np.ascontiguousarray(np.asarray(branch).reshape(npix), np.int64)
    bp = None if br is None else br.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    rc = L.oracle_backward(g.n, *[q for _, q in arrs], g.sh_degree, med[1], c[1], npix, pp, ptr(gout),
                           bp, float(near), int(bin), ptr(res["means"]), ptr(res["log_scales"]), ptr(res["quats"]), ptr(res["opacity_logits"]),
                           ptr(res["sh"]), ptr(res["medium"]), ptr(res["proj"]), nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_backward failed: {rc}")
    return res


def composite(alpha, col, d, medium, z_far):
    """The water model on one explicit front-to-back list (no skip or stop
    rules). Returns (rgb[3], T_after, D = sum d alpha T, A = sum alpha T)."""
    L = lib()
    alpha, pa = _d(alpha)
    col, pc = _d(np.asarray(col, np.float64).reshape(-1, 3))
    d, pd = _d(d)
    med, pm = _d(np.asarray(medium.as_array() if hasattr(medium, "as_array") else medium, np.float64))
    out = np.zeros(6)
    rc = L.oracle_composite(alpha.size, pa, pc, pd, pm, float(z_far), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("oracle_composite failed")
    return out[:3].copy(), out[3], out[4], out[5]


def sh_basis(deg: int, direction) -> np.ndarray:
    L = lib()
    d, pd = _d(direction)
    out = np.zeros((deg + 1) ** 2)
    rc = L.oracle_sh_basis(deg, pd, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise RuntimeError("bad degree")
    return out


def build() -> str:
    return _build.build()
