"""Oracle for the paper-literal pixel mode of the water model (Eq. 5), FP64.

TEST INFRASTRUCTURE ONLY (tests, smoke and the benchmark's CPU legs).

Eq. 5 applies the water once per pixel with the expected depth z of Eq. 6:
    C = J e^{-beta_D z} + B_inf (1 - e^{-beta_B z}),   J = sum_i c_i alpha_i T_i,
    z = (sum_i d_i alpha_i T_i) / (sum_i alpha_i T_i)   (z = z_far where nothing composites).
J and z are exactly what the segment-model oracle returns with a zero medium
(beta = 0, B_inf = 0 makes every effective colour the plain colour and removes
every backscatter term), with the same membership, skip and stop rules. The
adjoint follows by the chain rule through the same zero-medium adjoint:
    dL/dJ = G e^{-beta_D z}                       (G = dL/dC per channel)
    dL/dz += sum_ch G (B_inf beta_B e^{-beta_B z} - beta_D J e^{-beta_D z})   (only where sum alpha T > 0)
    dL/dbeta_D = sum_p -G z J e^{-beta_D z},  dL/dbeta_B = sum_p G B_inf z e^{-beta_B z},
    dL/dB_inf = sum_p G (1 - e^{-beta_B z}).
"""
from __future__ import annotations

import numpy as np

from . import backward as _seg_backward
from . import branches as _seg_branches
from . import render as _seg_render

ZERO = np.zeros(9)


def _split(medium):
    m = np.asarray(medium.as_array() if hasattr(medium, "as_array") else medium, np.float64)
    return m[0:3], m[3:6], m[6:9]


def _bcast(v, z):
    return np.asarray(v, np.float64).reshape((3,) + (1,) * z.ndim)


def _water(r, medium):
    bD, bB, binf = _split(medium)
    z = r["depth"]
    J = r["image"]
    a = np.exp(-_bcast(bD, z) * z)
    b = np.exp(-_bcast(bB, z) * z)
    out = dict(r)
    out["J"] = J
    out["image"] = J * a + _bcast(binf, z) * (1.0 - b)
    return out


def render(g, medium, cam, pix=None, nthreads: int = 0) -> dict:
    return _water(_seg_render(g, ZERO, cam, pix=pix, nthreads=nthreads), medium)


def branches(g, medium, cam, pix, nthreads: int = 0) -> dict:
    """The branches of the listed pixels' near decisions (see the segment
    oracle's ``branches``; the decisions do not depend on the medium), each
    with Eq. 5 applied."""
    return _water(_seg_branches(g, ZERO, cam, pix, nthreads=nthreads), medium)


def backward(g, medium, cam, dL_dimage, dL_ddepth=None, dL_ddepth01=None, pix=None, nthreads: int = 0,
             branch=None) -> dict:
    """``branch``: optional per-pixel branch of the near decisions (0 = the
    FP64 walk) whose J, z and adjoint are used."""
    r = _seg_render(g, ZERO, cam, pix=pix, nthreads=nthreads)
    bD, bB, binf = _split(medium)
    z, J, acc = r["depth"].copy(), r["image"].copy(), r["acc"].copy()
    if branch is not None and np.any(branch):
        bfl = np.asarray(branch).reshape(-1)
        idx = np.flatnonzero(bfl)
        lin = idx if pix is None else np.asarray(pix).reshape(-1)[idx]
        br = _seg_branches(g, ZERO, cam, lin, nthreads=nthreads)
        rows, pick = np.arange(idx.size), bfl[idx]
        z.reshape(-1)[idx] = br["depth"][rows, pick]
        J.reshape(3, -1)[:, idx] = br["image"][:, rows, pick]
        acc.reshape(-1)[idx] = (br["n_contrib"][rows, pick] > 0).astype(np.float64)
    G = np.asarray(dL_dimage, np.float64).reshape(J.shape)
    a = np.exp(-_bcast(bD, z) * z)
    b = np.exp(-_bcast(bB, z) * z)
    gJ = G * a
    dz = (G * (_bcast(binf, z) * _bcast(bB, z) * b - _bcast(bD, z) * J * a)).sum(0)
    dz = np.where(acc > 0, dz, 0.0)
    gz = dz + (np.asarray(dL_ddepth, np.float64).reshape(z.shape) if dL_ddepth is not None else 0.0)
    res = _seg_backward(g, ZERO, cam, gJ, dL_ddepth=gz, dL_ddepth01=dL_ddepth01, pix=pix, nthreads=nthreads,
                        branch=branch)
    axes = tuple(range(1, J.ndim))
    res["medium"] = np.concatenate([(-G * z * J * a).sum(axes), (G * _bcast(binf, z) * z * b).sum(axes),
                                    (G * (1.0 - b)).sum(axes)])
    return res
