"""Torch-facing API of the learned warm-start (argument marshalling only; the
featuriser, the GEMMs, the heads, the loss and Adam run in libsplash).

    rows = torch.empty((n, ROW), dtype=torch.bfloat16, device="cuda")
    featurise(renderer, image, depth, z_far, rows[i])     # one view -> one row
    net = Mlp(renderer, max_batch=256)
    net.set_params(scenes.mlp_init(seed))
    loss = net.step(rows, targets, idx, lr=1e-3)           # one Adam step
    pred = net.predict(rows[:k])                           # [k, 9] medium

Targets and predictions are the nine medium parameters (beta_D[3],
beta_B[3], B_inf[3]) in the renderer's medium layout.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi

IN, ROW, HIDDEN, OUT = _abi.MLP_IN, _abi.MLP_ROW, _abi.MLP_HIDDEN, _abi.MLP_OUT
SHAPES = {"W1": (HIDDEN, IN), "b1": (HIDDEN,), "W2": (HIDDEN, HIDDEN), "b2": (HIDDEN,), "W3": (OUT, HIDDEN),
          "b3": (OUT,)}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t: torch.Tensor, name: str, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def featurise(renderer, image: torch.Tensor, depth: torch.Tensor, z_far: float, row: torch.Tensor | None = None):
    """Feature row [ROW] (BF16) of one view: image [3,H,W] and metric depth [H,W]."""
    _need(image, "image", torch.float32)
    _need(depth, "depth", torch.float32)
    _, H, W = image.shape
    if tuple(depth.shape) != (H, W):
        raise ValueError("depth must be [H, W] of the image")
    if row is None:
        row = torch.empty(ROW, dtype=torch.bfloat16, device=image.device)
    _need(row, "row", torch.bfloat16, (ROW,))
    _abi.check(_abi.lib().splash_featurise(renderer._ctx, image.data_ptr(), depth.data_ptr(), W, H, float(z_far),
                                           row.data_ptr(), _stream()), "splash_featurise")
    return row


def gemm(renderer, A: torch.Tensor, B: torch.Tensor, D: torch.Tensor | None = None) -> torch.Tensor:
    """D = A B^T on the tensor cores (A [M,K], B [N,K] BF16; D [M,N] FP32)."""
    _need(A, "A", torch.bfloat16)
    _need(B, "B", torch.bfloat16)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must have the same K")
    if D is None:
        D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _need(D, "D", torch.float32, (M, N))
    _abi.check(_abi.lib().splash_gemm_bf16(renderer._ctx, A.data_ptr(), K, B.data_ptr(), K, D.data_ptr(), N, M, N, K,
                                           _stream()), "splash_gemm_bf16")
    return D


def _param_struct(p: dict) -> _abi.MlpParams:
    s = _abi.MlpParams()
    for k, shape in SHAPES.items():
        _need(p[k], k, torch.float32, shape)
        setattr(s, k, p[k].data_ptr())
    return s


class Mlp:
    """The 3080 -> 128 -> 128 -> 9 warm-start network (handle over libsplash)."""

    def __init__(self, renderer, max_batch: int = 256):
        self._renderer = renderer  # keeps the context alive
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().splash_mlp_create(renderer._ctx, int(max_batch), ctypes.byref(h)), "splash_mlp_create")
        self._h = h
        self.max_batch = int(max_batch)
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                torch.cuda.synchronize()
                _abi.lib().splash_mlp_destroy(h)
            except Exception:
                pass
            self._h = None

    def set_params(self, params: dict):
        """params: name -> array/tensor (FP32) with the shapes in SHAPES."""
        dev = {k: torch.as_tensor(np.asarray(params[k], np.float32) if not isinstance(params[k], torch.Tensor)
                                  else params[k], dtype=torch.float32).to("cuda").contiguous() for k in SHAPES}
        _abi.check(_abi.lib().splash_mlp_set_params(self._h, ctypes.byref(_param_struct(dev)), _stream()),
                   "splash_mlp_set_params")
        torch.cuda.current_stream().synchronize()

    def get_params(self) -> dict:
        out = {k: torch.empty(s, dtype=torch.float32, device="cuda") for k, s in SHAPES.items()}
        _abi.check(_abi.lib().splash_mlp_get_params(self._h, ctypes.byref(_param_struct(out)), _stream()),
                   "splash_mlp_get_params")
        return out

    def predict(self, rows: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        _need(rows, "rows", torch.bfloat16)
        if rows.dim() != 2 or rows.shape[1] != ROW:
            raise ValueError(f"rows must be [k, {ROW}]")
        k = rows.shape[0]
        if out is None:
            out = torch.empty((k, OUT), dtype=torch.float32, device=rows.device)
        _need(out, "out", torch.float32, (k, OUT))
        _abi.check(_abi.lib().splash_mlp_predict(self._h, rows.data_ptr(), k, out.data_ptr(), _stream()),
                   "splash_mlp_predict")
        return out

    def step(self, bank: torch.Tensor, targets: torch.Tensor, idx: torch.Tensor | None = None, batch: int | None = None,
             lr: float | None = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, grads: dict | None = None,
             loss: torch.Tensor | None = None) -> torch.Tensor:
        """One step on rows bank[idx] with targets[idx]; lr=None computes the
        loss (and ``grads`` if given) without updating. Returns the device loss."""
        _need(bank, "bank", torch.bfloat16)
        _need(targets, "targets", torch.float32)
        if bank.dim() != 2 or bank.shape[1] != ROW or targets.shape != (bank.shape[0], OUT):
            raise ValueError("bank must be [n, ROW] and targets [n, 9]")
        if idx is not None:
            _need(idx, "idx", torch.int32)
            batch = idx.shape[0]
        elif batch is None:
            batch = bank.shape[0]
        adam = None
        if lr is not None:
            adam = _abi.MlpAdam(float(lr), float(beta1), float(beta2), float(eps))
        g = None
        if grads is not None:
            for k, s in SHAPES.items():
                grads.setdefault(k, torch.empty(s, dtype=torch.float32, device="cuda"))
            g = _param_struct(grads)
        loss = self._loss if loss is None else loss
        _abi.check(_abi.lib().splash_mlp_step(self._h, bank.data_ptr(), bank.shape[0],
                                              idx.data_ptr() if idx is not None else None,
                                              targets.data_ptr(), int(batch),
                                              ctypes.byref(adam) if adam is not None else None, loss.data_ptr(),
                                              ctypes.byref(g) if g is not None else None, _stream()),
                   "splash_mlp_step")
        return loss
