"""Pins of the backscatter-estimate oracle (Sec. IV-B; Alg. 1 and Alg. 2)
against closed forms, invariants, hand-worked cases and brute force."""
import math

import numpy as np
import pytest

from oracle import backscatter as BS
from tests import water


# ------------------------------------------------------------------- resize
def test_resized_width():
    assert BS.resized_width(1920, 1280) == 450
    assert BS.resized_width(1280, 854) == 450   # 449.6 rounds up
    assert BS.resized_width(128, 96) == 400
    assert BS.resized_width(450, 300) == 450
    assert BS.resized_width(1, 5000) == 1       # never zero


def test_resize_same_height_is_identity():
    x = np.random.default_rng(0).uniform(0, 1, (3, 300, 451)).astype(np.float32)
    assert np.array_equal(BS.resize(x, 300), x)


def test_resize_integer_factor_is_block_mean():
    x = np.random.default_rng(1).uniform(0, 1, (3, 600, 800))
    want = x.reshape(3, 300, 2, 400, 2).mean(axis=(2, 4)).astype(np.float32)
    assert np.array_equal(BS.resize(x, 300), want)


@pytest.mark.parametrize("H,W,h", [(37, 53, 10), (854, 64, 300), (7, 9, 10), (96, 128, 300)])
def test_resize_equals_supersampled_block_mean(H, W, h):
    """Area averaging of a piecewise-constant image: replicate every source
    row h times and every column w times, then each output cell is the
    plain mean of an H x W block of the replicated grid."""
    x = np.random.default_rng(H + W).uniform(0, 1, (H, W))
    w = BS.resized_width(W, H, h)
    big = np.repeat(np.repeat(x, h, axis=0), w, axis=1)
    want = big.reshape(h, H, w, W).mean(axis=(1, 3)).astype(np.float32)
    np.testing.assert_array_max_ulp(BS.resize(x, h), want, maxulp=1)


def test_resize_preserves_mass_and_clamps():
    rng = np.random.default_rng(2)
    x = rng.uniform(0, 2, (1280, 1920))
    y = BS.resize(x, 300)
    assert math.isclose(y.astype(np.float64).sum() * (1280 * 1920) / (300 * 450), x.sum(), rel_tol=1e-6)
    neg = BS.resize(-np.abs(x), 300)
    assert np.all(neg == 0) and not np.any(np.signbit(neg))


# -------------------------------------------------------------- dark pixels
def test_dark_mask_hand_worked():
    """Depths 0..19 in one row; 10 edges over [0, 19] are 19 i / 9, so the
    clusters are {0,1,2}, {3,4}, {5,6}, ..., {15,16}, {17,18,19}. With
    p_dark = 0.5 the 3-pixel clusters keep 2 and the others keep 1. The
    colour of pixel j is chosen so that its rho is a known permutation."""
    z = np.arange(20, dtype=np.float32)[None]
    r = np.array([5, 1, 3, 9, 2, 4, 4, 7, 0, 8, 8, 6, 1, 2, 3, 9, 9, 0, 5, 1], np.float32)
    img = np.stack([r, np.zeros_like(r), np.zeros_like(r)])[:, None, :]
    keep, cl, _ = BS.dark_mask(img, z, p_dark=0.5)
    assert cl.tolist() == [0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5, 6, 6, 7, 7, 8, 8, 8]
    # c0: rho 5,1,3 -> pixels 1,2; c1: 9,2 -> 4; c2: tie 4,4 -> 5 (smaller index);
    # c3: 7,0 -> 8; c4: tie 8,8 -> 9; c5: 6,1 -> 12; c6: 2,3 -> 13;
    # c7: tie 9,9 -> 15; c8: 0,5,1 -> 17,19
    assert np.nonzero(keep)[0].tolist() == [1, 2, 4, 5, 8, 9, 12, 13, 15, 17, 19]


def test_two_bounds_make_one_bucket():
    """edges = 2 (or intervals = 2): a single cluster (interval) holds every pixel."""
    z = np.array([[3.0, 1.0, 2.0, 5.0]], np.float32)
    img = np.stack([np.array([[0.4, 0.3, 0.1, 0.2]], np.float32)] * 3)
    keep, cl, _ = BS.dark_mask(img, z, p_dark=0.5, edges=2)
    assert cl.tolist() == [0, 0, 0, 0] and np.nonzero(keep)[0].tolist() == [2, 3]
    pts = BS.depth_minima(img, z, np.ones(4, bool), intervals=2)
    assert all(p[0].tolist() == [2.0] for p in pts)


def test_dark_mask_constant_depth_is_one_top_cluster():
    img = np.random.default_rng(3).uniform(0, 1, (3, 10, 30)).astype(np.float32)
    z = np.full((10, 30), 4.0, np.float32)
    keep, cl, _ = BS.dark_mask(img, z)
    assert np.all(cl == 8)
    assert keep.sum() == math.ceil(0.01 * 300) == 3
    assert set(np.argsort(BS.rho(img).ravel(), kind="stable")[:3]) == set(np.nonzero(keep)[0])


def test_dark_mask_invariants_on_a_water_view():
    img, depth, _ = water.view(4, 1280, 854)
    img_s, z_s = BS.resize(img), BS.resize(depth[None])[0]
    keep, cl, e = BS.dark_mask(img_s, z_s)
    r = BS.rho(img_s).ravel()
    zf = z_s.ravel().astype(np.float64)
    # brute force of the cluster rule on every pixel
    assert np.array_equal(cl, [max(i for i in range(9) if zz >= e[i]) for zz in zf])
    for c in range(9):
        m = cl == c
        if not m.any():
            continue
        assert keep[m].sum() == math.ceil(0.01 * m.sum())
        if (~keep & m).any():
            assert r[keep & m].max() <= r[~keep & m].min()


# ------------------------------------------------------------ depth minima
def test_depth_minima_hand_worked():
    """Five kept pixels with depths 1, 2, 2.5, 4, 5; intervals = 3 gives
    bounds 1, 3, 5: interval 0 = {1, 2, 2.5}, interval 1 = {4, 5}."""
    z = np.array([[1.0, 2.0, 2.5, 4.0, 5.0, 9.0]], np.float32)
    img = np.array([[[0.3, 0.1, 0.2, 0.4, 0.4, 0.0]],
                    [[0.2, 0.5, 0.2, 0.9, 0.8, 0.0]],
                    [[0.7, 0.6, 0.5, 0.1, 0.2, 0.0]]], np.float32)
    keep = np.array([1, 1, 1, 1, 1, 0], bool)
    pts = BS.depth_minima(img, z, keep, intervals=3)
    f32 = lambda v: np.float64(np.float32(v))
    assert pts[0][0].tolist() == [2.0, 4.0] and pts[0][1].tolist() == [f32(0.1), f32(0.4)]  # tie 0.4/0.4 -> depth 4
    assert pts[1][0].tolist() == [1.0, 5.0] and pts[1][1].tolist() == [f32(0.2), f32(0.8)]  # tie 0.2/0.2 -> pixel 0
    assert pts[2][0].tolist() == [2.5, 4.0] and pts[2][1].tolist() == [f32(0.5), f32(0.1)]


# ---------------------------------------------------------------------- fit
ZS = np.linspace(1.0, 15.0, 24)


def test_fit_recovers_noise_free_model():
    for B, beta in [(0.3, 0.7), (0.05, 0.05), (0.9, 3.0), (0.2, 0.15)]:
        fb, fbeta, s = BS.fit_channel(ZS, B * (1 - np.exp(-beta * ZS)))
        assert abs(fb - B) < 1e-9 and abs(fbeta - beta) < 1e-8 and s < 1e-24


def test_fit_respects_bounds():
    m = 0.4 * (1 - np.exp(-7.0 * ZS))                                  # beta above 5
    fb, fbeta, _ = BS.fit_channel(ZS, m)
    f5 = 1 - np.exp(-5.0 * ZS)                                         # at beta = 5 the best B is linear LS
    assert fbeta <= 5.0 and abs(fbeta - 5.0) < 1e-9 and abs(fb - (m @ f5) / (f5 @ f5)) < 1e-9
    fb, fbeta, _ = BS.fit_channel(ZS, 1.4 * (1 - np.exp(-0.3 * ZS)))   # B above 1
    assert fb <= 1.0 and abs(fb - 1.0) < 1e-9
    fb, _, s = BS.fit_channel(ZS, np.zeros_like(ZS))
    assert fb == pytest.approx(0.0, abs=1e-12) and s == pytest.approx(0.0, abs=1e-24)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fit_is_the_global_minimum_over_a_dense_grid(seed):
    rng = np.random.default_rng(seed)
    B, beta = rng.uniform(0.05, 0.6), rng.uniform(0.05, 1.5)
    m = B * (1 - np.exp(-beta * ZS)) + rng.normal(0, 0.02, ZS.size)
    fb, fbeta, s = BS.fit_channel(ZS, m)
    gb, gbeta = np.meshgrid(np.linspace(0, 1, 401), np.linspace(0, 5, 2001), indexing="ij")
    pred = gb[..., None] * (1 - np.exp(-gbeta[..., None] * ZS))
    grid = ((m - pred) ** 2).sum(-1)
    assert s <= grid.min() + 1e-12          # no grid point does better
    assert s >= grid.min() - 1e-4           # and the grid comes close
    assert s == pytest.approx(BS.residual(fb, fbeta, ZS, m), rel=1e-12)


# --------------------------------------------------------------- end to end
def _recovery_view(seed, width, height):
    img, depth, med = water.view(seed, width, height, shadow_block=4, shadow_frac=0.04)
    return img, depth, med


def test_estimate_recovers_the_medium_when_shadows_are_pure_backscatter():
    """At 300 rows the resize is the identity; every cluster holds more
    shadow pixels than it keeps, so every fitted point lies on
    B_inf (1 - exp(-beta_B z)) and the fit returns the drawn medium."""
    img, depth, med = _recovery_view(5, 450, 300)
    est = BS.estimate(img, depth)
    np.testing.assert_allclose(est["binf"], med.b_inf, rtol=2e-5)
    np.testing.assert_allclose(est["beta_b"], med.beta_b, rtol=2e-5)
    assert all(len(z) >= 9 for z, _ in est["points"])


def test_estimate_invariant_under_exact_2x_downsample():
    img, depth, _ = _recovery_view(6, 450, 300)
    big_img = np.repeat(np.repeat(img, 2, axis=1), 2, axis=2)
    big_depth = np.repeat(np.repeat(depth, 2, axis=0), 2, axis=1)
    a, b = BS.estimate(img, depth), BS.estimate(big_img, big_depth)
    assert np.array_equal(a["keep"], b["keep"])
    assert np.array_equal(a["binf"], b["binf"]) and np.array_equal(a["beta_b"], b["beta_b"])


# ------------------------------------------------------------------ L_best
def test_prior_hand_worked():
    med = [0.5, 0.5, 0.5, 0.3, 0.2, 0.1, 0.2, 0.2, 0.2]
    loss, g = BS.prior_loss_and_grad(med, beta_b_hat=[0.1, 0.2, 0.5], binf_hat=[0.25, 0.1, 0.2], lam=0.1)
    assert loss == pytest.approx(0.1 * (0.2 + 0.0 + 0.4 + 0.05 + 0.1 + 0.0))
    assert np.allclose(g, 0.1 * np.array([0, 0, 0, 1, 0, -1, -1, 1, 0]))


def test_prior_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    med = rng.uniform(0.05, 0.6, 9)
    bh, Bh = rng.uniform(0.05, 0.6, 3), rng.uniform(0.05, 0.4, 3)
    _, g = BS.prior_loss_and_grad(med, bh, Bh)
    for j in range(9):
        e = np.zeros(9)
        e[j] = 1e-7
        fd = (BS.prior_loss_and_grad(med + e, bh, Bh)[0] - BS.prior_loss_and_grad(med - e, bh, Bh)[0]) / 2e-7
        assert fd == pytest.approx(g[j], abs=1e-6)
