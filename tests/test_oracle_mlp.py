"""Pins for the warm-start oracle (features, BF16 rounding, MLP and its
gradients) against library routines, closed forms and finite differences."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from paper_2411_19588_b300 import scenes


def test_bf16_round_matches_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7 + 2 ** -8, 65504.0, 3e38, -1e-40]])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16_round(x), ref)
    # ties go to even: 1 + 2^-8 sits halfway between 1 and 1 + 2^-7
    assert M.bf16_round(1 + 2 ** -8) == 1.0
    assert M.bf16_round(1 + 3 * 2 ** -8) == 1 + 2 ** -6
    np.testing.assert_array_equal(M.bf16_bits([1.0, -2.0]), [0x3F80, 0xC000])


@pytest.mark.parametrize("h,w", [(96, 128), (854, 1280), (33, 47), (32, 32), (40, 31)])
def test_downsample_is_adaptive_average_pool(h, w):
    img, _ = scenes.view_maps(1, w, h)
    ref = torch.nn.functional.adaptive_avg_pool2d(torch.tensor(img, dtype=torch.float64), (32, 32)).numpy()
    np.testing.assert_allclose(M.downsample(img), ref, rtol=1e-13, atol=1e-15)


def test_downsample_of_constant_and_of_exact_blocks():
    np.testing.assert_allclose(M.downsample(np.full((3, 50, 70), 0.37)), 0.37, rtol=1e-14)
    # 64x64 -> 2x2 blocks: brute force
    img = np.random.default_rng(2).uniform(0, 1, (3, 64, 64))
    ref = img.reshape(3, 32, 2, 32, 2).mean(axis=(2, 4))
    np.testing.assert_allclose(M.downsample(img), ref, rtol=1e-14)


def test_depth_histogram_closed_forms():
    zf = 20.0
    assert M.depth_histogram(np.full((10, 10), 3.0), zf).tolist() == [0, 1, 0, 0, 0, 0, 0, 0]
    # the far plane (empty pixels) and anything beyond fall in the last bin; negatives in the first
    assert M.depth_histogram(np.array([zf, 1e9, -1.0, 0.0]), zf).tolist() == [0.5, 0, 0, 0, 0, 0, 0, 0.5]
    # bin edges belong to the upper bin: k * 2.5 -> bin k
    assert M.depth_bin(np.arange(8) * 2.5, zf).tolist() == list(range(8))
    # a uniform ramp over [0, z_far) fills all bins equally
    z = (np.arange(800) + 0.5) * (zf / 800)
    np.testing.assert_allclose(M.depth_histogram(z, zf), np.full(8, 0.125))
    _, depth = scenes.view_maps(3, 128, 96)
    h = M.depth_histogram(depth, zf)
    # background (1/12 of the view at z_far) plus the uniform share of [17.5, 20): ~0.2
    assert abs(h.sum() - 1.0) < 1e-15 and 0.18 < h[7] < 0.22


def test_stored_feature_layout():
    img, depth = scenes.view_maps(4, 100, 60)
    row = M.stored_features(img, depth, 20.0)
    assert row.shape == (M.N_IN,)
    np.testing.assert_array_equal(row[:M.N_IMG], M.bf16_round(M.downsample(img).ravel()))
    np.testing.assert_array_equal(row[M.N_IMG:], M.bf16_round(M.depth_histogram(depth, 20.0)))
    # channel-major order: channel 1, cell (0, 0) averages rows 0..1, cols 0..3 of a 60x100 image
    assert row[1024] == M.bf16_round(img[1, 0:2, 0:4].mean())


def _torch_mlp(params, X, target, round_bf16):
    """The same network in torch FP64 with autograd; BF16 rounding by torch's
    own conversion with a straight-through gradient."""
    def rnd(t):
        if not round_bf16:
            return t
        return t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    x = rnd(torch.tensor(X, dtype=torch.float64))
    lin = lambda h, w, b: torch.nn.functional.linear(h, rnd(w), rnd(b))
    h1 = rnd(torch.relu(lin(x, P["W1"], P["b1"])))
    h2 = rnd(torch.relu(lin(h1, P["W2"], P["b2"])))
    h2.register_hook(lambda g: None)
    y = lin(h2, P["W3"], P["b3"])
    y.register_hook(lambda g: rnd(g))
    p = torch.cat([torch.nn.functional.softplus(y[:, :6]), torch.sigmoid(y[:, 6:])], 1)
    loss = torch.nn.functional.l1_loss(torch.log(p), torch.log(torch.tensor(target, dtype=torch.float64)))
    loss.backward()
    return loss.item(), {k: v.grad.numpy() for k, v in P.items()}, p.detach().numpy()


def _small_problem(seed, B=8):
    rng = np.random.default_rng(seed)
    params = scenes.mlp_init(seed)
    X = rng.uniform(0, 1, (B, M.N_IN))
    X[:, M.N_IMG:] = rng.dirichlet(np.ones(8), B)
    target = np.concatenate([rng.uniform(0.05, 0.6, (B, 6)), rng.uniform(0.05, 0.4, (B, 3))], 1)
    return params, X, target


def test_mlp_forward_and_grads_match_torch_autograd_fp64():
    params, X, target = _small_problem(5)
    loss, g, fw = M.loss_and_grads(params, X, target, round_bf16=False)
    tl, tg, tp = _torch_mlp(params, X, target, False)
    assert abs(loss - tl) < 1e-12
    np.testing.assert_allclose(M.heads(fw["Y"]), tp, rtol=1e-12)
    for k in g:
        np.testing.assert_allclose(g[k], tg[k], rtol=1e-9, atol=1e-14 * np.abs(tg[k]).max())


def test_mlp_rounded_forward_matches_torch_bf16_conversion():
    """With BF16 rounding: the forward values agree exactly with torch's
    conversion at the same points, and the backward signals other than the
    rounded dZ's agree (torch's hook rounds only dY, so compare W3, b3)."""
    params, X, target = _small_problem(6)
    loss, g, fw = M.loss_and_grads(params, X, target, round_bf16=True)
    tl, tg, tp = _torch_mlp(params, X, target, True)
    assert abs(loss - tl) < 1e-12
    np.testing.assert_allclose(M.heads(fw["Y"]), tp, rtol=1e-12)
    for k in ("W3", "b3"):
        np.testing.assert_allclose(g[k], tg[k], rtol=1e-9, atol=1e-14 * np.abs(tg[k]).max())


def test_mlp_grads_match_central_differences():
    """FP64 central differences of the unrounded loss at a few coordinates of
    every parameter (kinks of |.| and ReLU avoided by the random point)."""
    params, X, target = _small_problem(7, B=4)
    p64 = {k: v.astype(np.float64) for k, v in params.items()}
    _, g, _ = M.loss_and_grads(p64, X, target, round_bf16=False)
    rng = np.random.default_rng(8)
    for k, v in p64.items():
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in v.shape)
            h = 1e-6 * max(1.0, abs(v[idx]))
            vp, vm = dict(p64), dict(p64)
            vp[k] = v.copy(); vp[k][idx] += h
            vm[k] = v.copy(); vm[k][idx] -= h
            fd = (M.loss_and_grads(vp, X, target, False)[0] - M.loss_and_grads(vm, X, target, False)[0]) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-6 * max(1e-3, abs(fd)), (k, idx, fd, g[k][idx])


def test_heads_closed_forms():
    y = np.zeros((1, 9))
    np.testing.assert_allclose(M.heads(y), [[np.log(2)] * 6 + [0.5] * 3])
    # prediction equal to the target: zero loss
    y = np.array([[-0.957] * 6 + [-1.237] * 3])
    loss, dY = M.loss_and_dy(y, M.heads(y))
    assert loss == 0.0 and not dY.any()


def test_gemm_nt_brute_force():
    rng = np.random.default_rng(9)
    A, B = rng.standard_normal((5, 7)), rng.standard_normal((3, 7))
    ref = np.array([[sum(A[i, k] * B[j, k] for k in range(7)) for j in range(3)] for i in range(5)])
    np.testing.assert_allclose(M.gemm_nt(A, B), ref, rtol=1e-13)
