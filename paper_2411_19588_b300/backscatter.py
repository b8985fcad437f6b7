"""Torch-facing API of the backscatter estimate and the L_best prior
(Sec. IV-B, Eq. 7-9; appendix Alg. 1 and Alg. 2): argument marshalling for
splash_backscatter_estimate and splash_backscatter_prior; every step runs in
libsplash.

    res = estimate(renderer, target_image, depth)      # device result record
    prior = prior_of(res)                              # float32[6] view: beta_B_hat, B_inf_hat
    renderer.backward_adam(..., prior=prior, lambda_est=0.1)
    read(res)                                          # host dict (synchronises)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

RESULT_BYTES = ctypes.sizeof(_abi.BackscatterResult)
DEFAULTS = {"resized_height": 300, "edges": 10, "intervals": 25, "p_dark": 0.01, "b_max": 1.0, "beta_max": 5.0}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def options(**kw) -> _abi.BackscatterOptions:
    o = dict(DEFAULTS)
    o.update(kw)
    return _abi.BackscatterOptions(int(o["resized_height"]), int(o["edges"]), int(o["intervals"]), 0,
                                   float(o["p_dark"]), float(o["b_max"]), float(o["beta_max"]))


def resized_size(width: int, height: int, resized_height: int = 300) -> tuple[int, int]:
    """(w, h) of the resized maps."""
    return max(1, (2 * width * resized_height + height) // (2 * height)), resized_height


def new_result() -> torch.Tensor:
    return torch.zeros(RESULT_BYTES, dtype=torch.uint8, device="cuda")


def estimate(renderer, image: torch.Tensor, depth: torch.Tensor, result: torch.Tensor | None = None,
             resized: torch.Tensor | None = None, dark: torch.Tensor | None = None, **opts) -> torch.Tensor:
    """Estimate from an observed image [3,H,W] and the expected depth [H,W]
    of the current scene at the same view. Returns the device result record
    (uint8[RESULT_BYTES]). resized ([4,h,w] float32) and dark ([h,w] uint8)
    optionally receive the resized maps and the kept-pixel mask."""
    _need(image, "image", torch.float32)
    if image.dim() != 3 or image.shape[0] != 3:
        raise ValueError("image must be [3,H,W]")
    H, W = image.shape[1:]
    _need(depth, "depth", torch.float32, (H, W))
    o = options(**opts)
    w, h = resized_size(W, H, o.resized_height)
    if result is None:
        result = new_result()
    _need(result, "result", torch.uint8, (RESULT_BYTES,))
    if resized is not None:
        _need(resized, "resized", torch.float32, (4, h, w))
    if dark is not None:
        _need(dark, "dark", torch.uint8, (h, w))
    rc = _abi.lib().splash_backscatter_estimate(renderer._ctx, image.data_ptr(), depth.data_ptr(), int(W), int(H),
                                                ctypes.byref(o), result.data_ptr(), _abi.ptr(resized), _abi.ptr(dark),
                                                _stream())
    _abi.check(rc, "splash_backscatter_estimate")
    return result


def prior_of(result: torch.Tensor) -> torch.Tensor:
    """The first six floats of a result record (beta_B_hat[3], B_inf_hat[3]),
    aligned with medium[3:9]."""
    return result[:24].view(torch.float32)


def read(result: torch.Tensor) -> dict:
    """Host copy of a result record."""
    raw = result.cpu().numpy().tobytes()
    r = _abi.BackscatterResult.from_buffer_copy(raw)
    npts = list(r.n_points)
    return {"beta_b": np.array(r.beta_b[:], np.float32), "b_inf": np.array(r.b_inf[:], np.float32),
            "residual": np.array(r.residual[:], np.float32), "n_points": npts, "n_dark": r.n_dark,
            "width": r.width, "height": r.height,
            "points": [(np.array(r.point_z[k][:npts[k]], np.float32), np.array(r.point_v[k][:npts[k]], np.float32))
                       for k in range(3)]}


def prior(medium: torch.Tensor, prior_vec: torch.Tensor, lambda_est: float = 0.1, grad_medium=None, loss=None):
    """Adds Eq. 9's lambda_est L_best to *loss and its gradient to
    grad_medium[3:9] (device tensors, either may be None)."""
    _need(medium, "medium", torch.float32, (9,))
    _need(prior_vec, "prior", torch.float32, (6,))
    if grad_medium is not None:
        _need(grad_medium, "grad_medium", torch.float32, (9,))
    if loss is not None:
        _need(loss, "loss", torch.float32, (1,))
    rc = _abi.lib().splash_backscatter_prior(medium.data_ptr(), prior_vec.data_ptr(), float(lambda_est),
                                             _abi.ptr(grad_medium), _abi.ptr(loss), _stream())
    _abi.check(rc, "splash_backscatter_prior")
