"""Oracle for the learned warm-start: view features and the BF16 MLP, FP64 numpy.

TEST INFRASTRUCTURE ONLY (tests, smoke and the benchmark's CPU legs). The
paper has no learned component; this form predicts the nine per-channel
medium parameters of Eq. 4-5 (beta_D, beta_B, B_inf) from one rendered view
so that the fit of Sec. IV-C can start from them.

Definitions (each is the plain statement of what the CUDA path computes):

* Features of a view (image [3,H,W], expected depth z [H,W] from Eq. 6):
  - a 32x32 adaptive-average downsample per colour channel: output cell
    (i, j) averages rows floor(i H/32) .. ceil((i+1) H/32)-1 and columns
    floor(j W/32) .. ceil((j+1) W/32)-1 with equal weights;
  - an 8-bin histogram of z over [0, z_far]: bin = floor(fl32(fl32(8 z) /
    z_far)) clamped to [0, 7] (the integer decision is taken in FP32 on
    both sides), divided by H W;
  - order: [channel][i][j] (3072 values), then the 8 bins; stored as BF16.
* MLP 3080 -> 128 -> 128 -> 9 with ReLU hidden layers. Every weight matrix
  carries its bias as one more input column that multiplies a constant 1.
  Weights are FP32 masters used as BF16 copies; products are summed in
  FP32 (here FP64); the hidden activations H1, H2 and the backward signals
  dY, dZ2, dZ1 are rounded to BF16 where the GPU stores them.
* Heads: beta = softplus(y[0:6]), B_inf = sigmoid(y[6:9]).
* Loss: mean over the batch and the 9 outputs of |log p_hat - log p|.
  Backward treats BF16 rounding as the identity (straight-through) and takes
  d|u|/du = sign(u) with sign(0) = 0.

BF16 rounding: an FP64 value is rounded to FP32 (nearest even), then to the
nearest BF16 (the upper 16 bits of the FP32 pattern, ties to even).
"""
from __future__ import annotations

import math

import numpy as np

GRID = 32
N_BINS = 8
N_IMG = 3 * GRID * GRID          # 3072
N_IN = N_IMG + N_BINS            # 3080 features
HID = 128
N_OUT = 9


# ---------------------------------------------------------------------- BF16
def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (via FP32, ties to even), as float64."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    finite = np.isfinite(f)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    r = np.where(finite, r, u & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def bf16_bits(x) -> np.ndarray:
    """The 16-bit patterns of bf16_round(x)."""
    return (bf16_round(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


# ------------------------------------------------------------------ features
def _bounds(i: int, n: int):
    return (i * n) // GRID, -((-(i + 1) * n) // GRID)


def downsample(image) -> np.ndarray:
    """[3, 32, 32] adaptive averages of image [3, H, W], FP64."""
    img = np.asarray(image, np.float64)
    _, H, W = img.shape
    out = np.empty((3, GRID, GRID))
    for i in range(GRID):
        y0, y1 = _bounds(i, H)
        for j in range(GRID):
            x0, x1 = _bounds(j, W)
            out[:, i, j] = img[:, y0:y1, x0:x1].mean(axis=(1, 2))
    return out


def depth_bin(z, z_far) -> np.ndarray:
    """Histogram bin of each depth, decided in FP32."""
    z32 = np.asarray(z, np.float32)
    t = (z32 * np.float32(N_BINS)) / np.float32(z_far)
    b = np.floor(t.astype(np.float32))
    return np.clip(np.nan_to_num(b, nan=N_BINS - 1), 0, N_BINS - 1).astype(np.int64)


def depth_histogram(depth, z_far) -> np.ndarray:
    d = np.asarray(depth)
    counts = np.bincount(depth_bin(d.ravel(), z_far), minlength=N_BINS)
    return counts / float(d.size)


def features(image, depth, z_far) -> np.ndarray:
    """FP64 feature vector [3080] of one view (before BF16 storage)."""
    return np.concatenate([downsample(image).ravel(), depth_histogram(depth, z_far)])


def stored_features(image, depth, z_far) -> np.ndarray:
    """The stored feature vector [3080]: the features rounded to BF16."""
    return bf16_round(features(image, depth, z_far))


# ----------------------------------------------------------------------- MLP
def _softplus(y):
    return np.where(y > 20, y, np.log1p(np.exp(np.minimum(y, 20))))


def _sigmoid(y):
    return 1.0 / (1.0 + np.exp(-y))


def heads(y):
    """Predicted parameters [B, 9] from the network outputs y [B, 9]."""
    y = np.asarray(y, np.float64)
    return np.concatenate([_softplus(y[:, :6]), _sigmoid(y[:, 6:])], axis=1)


def forward(params: dict, X, round_bf16: bool = True) -> dict:
    """params: W1 [128,3080], b1 [128], W2 [128,128], b2, W3 [9,128], b3
    (FP32 masters). X: [B, 3080] feature values. Returns the intermediates."""
    rnd = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3 = (rnd(params[k]) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (rnd(params[k]) for k in ("b1", "b2", "b3"))
    X = rnd(X)
    Z1 = X @ W1.T + b1
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = rnd(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + b3
    return {"X": X, "W1": W1, "W2": W2, "W3": W3, "H1": H1, "H2": H2, "Y": Y}


def loss_and_dy(Y, target):
    """Mean |log heads(Y) - log target| and its derivative w.r.t. Y."""
    Y = np.asarray(Y, np.float64)
    t = np.asarray(target, np.float64)
    B = Y.shape[0]
    p = heads(Y)
    u = np.log(p) - np.log(t)
    loss = np.abs(u).sum() / (B * N_OUT)
    dlogp = np.concatenate([_sigmoid(Y[:, :6]) / p[:, :6], 1.0 - p[:, 6:]], axis=1)
    dY = np.sign(u) * dlogp / (B * N_OUT)
    return loss, dY


def backward(fw: dict, dY, round_bf16: bool = True) -> dict:
    """Gradients of the loss w.r.t. the masters, given dL/dY."""
    rnd = bf16_round if round_bf16 else (lambda a: np.asarray(a, np.float64))
    dY = rnd(dY)
    g = {"W3": dY.T @ fw["H2"], "b3": dY.sum(0)}
    dZ2 = rnd((dY @ fw["W3"]) * (fw["H2"] > 0))
    g["W2"], g["b2"] = dZ2.T @ fw["H1"], dZ2.sum(0)
    dZ1 = rnd((dZ2 @ fw["W2"]) * (fw["H1"] > 0))
    g["W1"], g["b1"] = dZ1.T @ fw["X"], dZ1.sum(0)
    return g


def loss_and_grads(params: dict, X, target, round_bf16: bool = True):
    fw = forward(params, X, round_bf16)
    loss, dY = loss_and_dy(fw["Y"], target)
    return loss, backward(fw, dY, round_bf16), fw


def predict(params: dict, X, round_bf16: bool = True) -> np.ndarray:
    return heads(forward(params, X, round_bf16)["Y"])


def gemm_nt(A, B) -> np.ndarray:
    """D = A B^T in FP64 (A [M,K], B [N,K])."""
    return np.asarray(A, np.float64) @ np.asarray(B, np.float64).T
