"""The learned warm-start on the GPU against the oracle: the tensor-core GEMM,
the featuriser, and the MLP's predictions, gradients and Adam step."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import adam as oadam
from oracle import mlp as O
from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import mlp as M
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r(cuda_lib):
    return R.Renderer()


def _bf16(rng, shape, scale=1.0):
    """Seeded BF16 input (torch's conversion) and its exact values in FP64."""
    t = torch.tensor(rng.standard_normal(shape) * scale, dtype=torch.float32).to(torch.bfloat16)
    return t.cuda(), t.to(torch.float64).numpy()


@pytest.mark.parametrize("M_,N_,K_", [(128, 16, 64), (256, 128, 3136), (128, 3136, 256), (384, 208, 192),
                                      (128, 256, 1024), (512, 48, 640), (2048, 2560, 128)])
def test_gemm_matches_fp64(r, M_, N_, K_):
    rng = np.random.default_rng(M_ + N_ + K_)
    A, a = _bf16(rng, (M_, K_))
    B, b = _bf16(rng, (N_, K_))
    D = M.gemm(r, A, B)
    r.sync_status()
    ref = O.gemm_nt(a, b)
    bound = 4 * K_ * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    err = np.abs(D.cpu().numpy() - ref)
    assert (err <= bound).all(), (err / bound).max()


def test_gemm_leading_dimensions_and_rejections(r):
    rng = np.random.default_rng(11)
    A, a = _bf16(rng, (128, 256))
    B, b = _bf16(rng, (64, 256))
    D = torch.full((128, 80), -7.0, device="cuda")
    L = _abi.lib()
    # K = 192 of the 256 stored columns; D written into the first 64 of 80 columns
    _abi.check(L.splash_gemm_bf16(r._ctx, A.data_ptr(), 256, B.data_ptr(), 256, D.data_ptr(), 80, 128, 64, 192,
                                  R._stream()), "gemm")
    r.sync_status()
    np.testing.assert_allclose(D[:, :64].cpu().numpy(), O.gemm_nt(a[:, :192], b[:, :192]), rtol=1e-5, atol=1e-4)
    assert (D[:, 64:] == -7.0).all()
    for m, n, k in [(100, 64, 192), (128, 24, 192), (128, 64, 100), (0, 64, 64)]:
        assert L.splash_gemm_bf16(r._ctx, A.data_ptr(), 256, B.data_ptr(), 256, D.data_ptr(), 80, m, n, k,
                                  R._stream()) == _abi.ERR_INVALID_ARG


@pytest.mark.parametrize("w,h", [(128, 96), (1280, 854), (47, 33), (20, 10), (1920, 1280)])
def test_featurise_matches_oracle(r, w, h):
    img, depth = scenes.view_maps(w * 7 + h, w, h)
    row = M.featurise(r, torch.tensor(img, device="cuda"), torch.tensor(depth, device="cuda"), 20.0)
    r.sync_status()
    got = row.float().cpu().numpy().astype(np.float64)
    # the stored row's layout: the 3080 features, the bias input 1, zeros to the padded width
    ref = np.zeros(M.ROW)
    ref[:O.N_IN] = O.stored_features(img, depth, 20.0)
    ref[O.N_IN] = 1.0
    assert got.shape == (M.ROW,)
    # histogram, bias input and padding: decided in FP32 on both sides, bit-exact
    np.testing.assert_array_equal(got[O.N_IMG:], ref[O.N_IMG:])
    # cell means: equal BF16 unless the FP64 mean sits within 1e-5 (relative) of a rounding midpoint
    mean = O.downsample(img).ravel()
    lo = O.bf16_round(mean * (1 - 1e-5))
    hi = O.bf16_round(mean * (1 + 1e-5))
    near = lo != hi
    assert near.mean() < 0.01
    np.testing.assert_array_equal(got[:O.N_IMG][~near], ref[:O.N_IMG][~near])
    assert np.isin(got[:O.N_IMG][near], np.stack([lo[near], hi[near]])).all() or near.sum() == 0


def _bank(seed, n):
    """Seeded feature rows (BF16 via torch's conversion) with the bias input, and targets."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n, M.ROW), np.float32)
    x[:, :O.N_IMG] = rng.uniform(0, 1, (n, O.N_IMG))
    x[:, O.N_IMG:O.N_IN] = rng.dirichlet(np.ones(8), n)
    x[:, O.N_IN] = 1.0
    xb = torch.tensor(x).to(torch.bfloat16)
    t = np.concatenate([rng.uniform(0.05, 0.6, (n, 6)), rng.uniform(0.05, 0.4, (n, 3))], 1).astype(np.float32)
    return xb.cuda(), xb.to(torch.float64).numpy()[:, :O.N_IN], torch.tensor(t).cuda(), t.astype(np.float64)


def test_predict_matches_oracle(r):
    params = scenes.mlp_init(3)
    net = M.Mlp(r, 256)
    net.set_params(params)
    bank, x, _, _ = _bank(4, 300)
    for k in (256, 37, 1):
        pred = net.predict(bank[:k].contiguous())
        r.sync_status()
        ref = O.predict(params, x[:k])
        np.testing.assert_allclose(pred.cpu().numpy(), ref, rtol=1e-3, atol=1e-6)


def _grads(net, bank, targets, idx):
    g = {}
    loss = net.step(bank, targets, idx=idx, lr=None, grads=g)
    torch.cuda.synchronize()
    return loss.item(), {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def _check_grads(got, ref):
    for k in ref:
        scale = np.abs(ref[k]).max()
        err = np.abs(got[k] - ref[k])
        # BF16 rounding of dY, dZ2, dZ1 on both sides: an element whose FP32 and
        # FP64 values straddle a BF16 rounding boundary moves by one BF16 ulp
        assert (err <= 1e-2 * np.abs(ref[k]) + 2e-3 * scale).all(), (k, (err / scale).max())
        assert np.median(err / (np.abs(ref[k]) + 1e-12 * scale)) < 1e-3, k


def test_gradients_match_oracle_and_padding_rows_are_clean(r):
    params = scenes.mlp_init(5)
    net = M.Mlp(r, 256)
    net.set_params(params)
    bank, x, tg, t = _bank(6, 500)
    rng = np.random.default_rng(7)
    # a full batch first, then a short one (rows past the batch must not leak)
    for B in (256, 37, 130):
        idx = np.sort(rng.choice(500, B, replace=False)).astype(np.int32)
        loss, got = _grads(net, bank, tg, torch.tensor(idx).cuda())
        r.sync_status()
        rl, rg, _ = O.loss_and_grads(params, x[idx], t[idx])
        assert abs(loss - rl) <= 1e-4 * rl
        _check_grads(got, rg)


def test_adam_step_matches_oracle(r):
    params = scenes.mlp_init(8)
    net = M.Mlp(r, 256)
    net.set_params(params)
    bank, x, tg, t = _bank(9, 256)
    lr = 1e-3
    net.step(bank, tg, lr=lr, eps=1e-8)
    after = {k: v.cpu().numpy().astype(np.float64) for k, v in net.get_params().items()}
    r.sync_status()
    _, g, _ = O.loss_and_grads(params, x, t)
    for k in params:
        p1, _, _ = oadam.adam_step(params[k], g[k], np.zeros_like(g[k]), np.zeros_like(g[k]), 1, lr, eps=1e-8)
        firm = np.abs(g[k]) > 1e-2 * np.abs(g[k]).max()
        np.testing.assert_allclose(after[k][firm], p1[firm], rtol=0, atol=1e-6)
        # elsewhere the first Adam step is lr * sign(g): at most the sign can differ
        assert (np.abs(after[k] - p1) <= 2 * lr + 1e-6).all()


def test_training_reduces_loss(r):
    params = scenes.mlp_init(10)
    net = M.Mlp(r, 256)
    net.set_params(params)
    bank, _, tg, _ = _bank(11, 1024)
    # make the targets a learnable function of the features
    tg[:, :] = 0.05 + 0.5 * bank[:, :9].float()
    gen = torch.Generator(device="cuda").manual_seed(0)
    held = torch.arange(0, 1024, 4, dtype=torch.int32, device="cuda")
    first = net.step(bank, tg, idx=held, lr=None).item()
    for _ in range(300):
        idx = torch.randint(0, 1024, (256,), device="cuda", generator=gen, dtype=torch.int32)
        net.step(bank, tg, idx=idx, lr=1e-3)
    last = net.step(bank, tg, idx=held, lr=None).item()
    r.sync_status()
    assert last < 0.5 * first, (first, last)


def test_out_of_range_rows_are_clamped_and_reported(r):
    net = M.Mlp(r, 128)
    net.set_params(scenes.mlp_init(12))
    bank, _, tg, _ = _bank(13, 64)
    idx = torch.tensor([0, 5, 64, -3], dtype=torch.int32, device="cuda")
    net.step(bank, tg, idx=idx, lr=None)
    with pytest.raises(_abi.SplashError) as ei:
        r.sync_status()
    assert ei.value.status == _abi.ERR_INVALID_ARG
    # the context still works
    net.step(bank, tg, idx=idx[:2].contiguous(), lr=None)
    r.sync_status()
