"""Pins of the oracle's near-decision branches (CPU only).

A decision whose FP64 quantity lies within oracle.NEAR of its threshold may
be taken either way by an FP32 evaluation of the definition; the oracle's
``branches`` renders the pixel with it taken the other way. Each case below
places one decision 5e-6 (relative) on one side of its threshold and checks
that the flipped branch equals the plain render of the same scene nudged
5e-6 across the threshold: a different scene, rendered by the ordinary
walk, whose only discrete difference is that decision. The nudge moves
the continuous result by far less than the 1e-6 compared here. Decisions:
the 3-sigma cut (Sec. III-A, "several standard deviations"), the alpha
skip and the transmittance stop (the 3DGS rules the paper keeps, Sec.
IV-D) and the depth order of Eq. 1 at FP32 resolution.
"""
import math

import numpy as np

import oracle
from paper_2411_19588_b300 import scenes

EPS = 5e-6
W = H = 64
F = 100.0
MED = scenes.Medium(np.float32([0.4, 0.2, 0.1]), np.float32([0.3, 0.25, 0.2]), np.float32([0.05, 0.2, 0.3]))


def _cam(R=np.eye(3), cx=32.0, cy=32.0):
    return scenes.Camera(W, H, F, F, cx, cy, np.concatenate([R, np.zeros((3, 1))], 1), 0.2, 20.0)


def _scene(means, log_scales, logits, rgb):
    n = len(means)
    sh = ((np.asarray(rgb, np.float64) - 0.5) / 0.28209479177387814).reshape(n, 1, 3)
    return scenes.Gaussians(np.float32(means), np.float32(np.repeat(np.asarray(log_scales, np.float64)[:, None], 3, 1)),
                            np.tile(np.float32([1, 0, 0, 0]), (n, 1)), np.float32(logits), np.float32(sh), 0)


def _logit(p):
    return math.log(p / (1.0 - p))


def _check(g_near, g_nudged, cam, pix, kind_note, nudged_near=1):
    near = oracle.render(g_near, MED, cam, pix=[pix])
    assert near["n_near"][0] == 1, (kind_note, near["n_near"][0], near["margin"][0])
    br = oracle.branches(g_near, MED, cam, [pix])
    assert br["valid"][0, :2].all() and not br["valid"][0, 2:].any()
    # branch 0 is the plain render
    np.testing.assert_array_equal(br["image"][:, 0, 0], near["image"][:, 0])
    assert br["depth"][0, 0] == near["depth"][0]
    nudged = oracle.render(g_nudged, MED, cam, pix=[pix])
    assert nudged["n_near"][0] == nudged_near
    np.testing.assert_allclose(br["image"][:, 0, 1], nudged["image"][:, 0], atol=1e-6, err_msg=kind_note)
    np.testing.assert_allclose(br["depth"][0, 1], nudged["depth"][0], rtol=1e-6, err_msg=kind_note)
    assert br["n_contrib"][0, 1] == nudged["n_contrib"][0]
    # the flip is visible: the two branches differ far beyond the image tolerance
    assert np.abs(br["image"][:, 0, 1] - br["image"][:, 0, 0]).max() > 1e-4, kind_note
    # the adjoint of the flipped branch is the adjoint of the nudged scene
    G = np.array([[0.7], [-0.4], [1.1]])
    a = oracle.backward(g_near, MED, cam, G, np.array([0.05]), np.array([0.3]), pix=[pix], branch=[1])
    b = oracle.backward(g_nudged, MED, cam, G, np.array([0.05]), np.array([0.3]), pix=[pix])
    for k in ("means", "log_scales", "opacity_logits", "sh", "medium"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-4, atol=1e-7 * max(1.0, np.abs(b[k]).max()), err_msg=k)
    return near, br


def _cut_scene(eps):
    # isotropic Gaussian on the axis at z = 3; pixel (40, 32) sees dx = 8.5, dy = 0.5
    z, r2 = 3.0, 8.5 ** 2 + 0.5 ** 2
    k = 9.0 * (1.0 + eps) / r2            # conic 1 / (s^2 f^2 / z^2 + 0.3) giving q = 9 (1 + eps)
    s = math.sqrt(1.0 / k - 0.3) * z / F
    return _scene([[0.0, 0.0, z]], [math.log(s)], [2.0], [[0.9, 0.3, 0.6]])


def test_cut_branch_equals_the_nudged_scene():
    pix = 32 * W + 40
    near, br = _check(_cut_scene(EPS), _cut_scene(-EPS), _cam(), pix, "3-sigma cut")
    assert near["n_contrib"][0] == 0 and br["n_contrib"][0, 1] == 1


def _skip_scene(eps):
    # centre on the pixel centre (32.5, 32.5): alpha = sigmoid(o) = (1/255)(1 + eps)
    return _scene([[0.0, 0.0, 3.0]], [-3.0], [_logit((1.0 + eps) / 255.0)], [[0.9, 0.3, 0.6]])


def test_skip_branch_equals_the_nudged_scene():
    pix = 32 * W + 32
    near, br = _check(_skip_scene(-EPS), _skip_scene(EPS), _cam(cx=32.5, cy=32.5), pix, "alpha skip")
    assert near["n_contrib"][0] == 0 and br["n_contrib"][0, 1] == 1


def _stop_scene(eps):
    # two in front at alpha 0.97 (T = 9e-4 behind them); the third with
    # 9e-4 (1 - alpha_c) = 1e-4 (1 + eps); a fourth behind all of them
    ac = 1.0 - 1e-4 * (1.0 + eps) / 9e-4
    return _scene([[0.0, 0.0, 2.0], [0.0, 0.0, 2.5], [0.0, 0.0, 3.0], [0.0, 0.0, 4.0]], [-3.0] * 4,
                  [_logit(0.97), _logit(0.97), _logit(ac), _logit(0.5)],
                  [[0.9, 0.3, 0.6], [0.2, 0.8, 0.4], [0.5, 0.5, 0.9], [0.1, 0.9, 0.9]])


def test_stop_branch_equals_the_nudged_scene():
    pix = 32 * W + 32
    near, br = _check(_stop_scene(-EPS), _stop_scene(EPS), _cam(cx=32.5, cy=32.5), pix, "transmittance stop")
    assert near["n_contrib"][0] == 2 and br["n_contrib"][0, 1] == 3


def test_order_branch_equals_the_nudged_scene():
    """Two Gaussians whose camera-frame depths round to one float, the
    nearer one with the higher index: the FP32 order (ties to the lower
    index) puts the farther one first. The camera turns by 1e-7 rad about
    y, so depth = cos(t) z - sin(t) x separates means 0.4 m apart in x by
    4e-8 m, below half an FP32 ulp at 3 m."""
    t = 1e-7
    R = np.array([[math.cos(t), 0, math.sin(t)], [0, 1, 0], [-math.sin(t), 0, math.cos(t)]])
    cam = _cam(R, cx=32.5, cy=32.5)

    def scene(z0):
        # index 0 at x = 0, index 1 at x = 0.4 (nearer by 4e-8 m when z0 = 3)
        return _scene([[0.0, 0.0, z0], [0.4, 0.0, 3.0]], [-1.0, -1.0], [0.0, 0.5],
                      [[0.9, 0.3, 0.6], [0.1, 0.7, 0.2]])

    P = oracle.project(scene(3.0), MED, cam)
    assert P["d"][1] < P["d"][0] and np.float32(P["d"][1]) == np.float32(P["d"][0])
    pix = 32 * W + 34
    # nudged: index 0 moves 1e-6 m nearer, so the exact order is the index
    # order and no near decision is left
    near, br = _check(scene(3.0), scene(3.0 - 1e-6), cam, pix, "FP32 depth order", nudged_near=0)
    assert near["tie"][0] == 1


def test_branch_zero_is_the_plain_render_everywhere():
    g, m, cam = scenes.tiny_scene(0)
    r = oracle.render(g, m, cam)
    pix = np.arange(0, cam.width * cam.height, 37)
    br = oracle.branches(g, m, cam, pix)
    np.testing.assert_array_equal(br["image"][:, :, 0], r["image"].reshape(3, -1)[:, pix])
    np.testing.assert_array_equal(br["depth"][:, 0], r["depth"].reshape(-1)[pix])
    nn = r["n_near"].reshape(-1)[pix]
    np.testing.assert_array_equal(br["valid"].sum(1), np.where(nn <= 4, 2 ** nn, 1))


def test_near_decisions_are_rare_at_the_tolerance():
    """The density of near decisions on the tiny workload: the exclusion
    budget of the comparison (0.1 %) is never approached because every
    pixel with at most four near decisions is compared on its branches."""
    g, m, cam = scenes.tiny_scene(0)
    r = oracle.render(g, m, cam)
    assert (r["n_near"] > 4).sum() == 0
    assert (r["n_near"] > 0).mean() < 1e-3


def test_binned_scan_equals_the_full_scan():
    """The binned candidate scan (bin x bin pixel blocks, widened 3-sigma
    boxes) gives the unbinned oracle's results bit for bit: images, depths,
    decision margins, near-decision counts, branches and gradients, on the
    tiny workload and on a dense ragged scene with large Gaussians."""
    rng = np.random.default_rng(4)
    g, m, cam = scenes.tiny_scene(0)
    cases = [(g, m, cam, 16), (g, m, cam, 7)]
    n = 1500
    cam2 = scenes.look_at((0.2, -0.1, -0.3), (0.0, 0.0, 3.5), 91, 67, 80.0, 80.0)
    g2 = scenes.Gaussians(np.float32(np.c_[rng.uniform(-1.5, 1.5, (n, 2)), rng.uniform(1.5, 6.0, n)]),
                          np.float32(rng.normal(-1.8, 0.6, (n, 3))), np.float32(rng.standard_normal((n, 4))),
                          np.float32(rng.normal(0.5, 1.0, n)), np.float32(rng.normal(0, 0.3, (n, 4, 3))), 1)
    cases.append((g2, m, cam2, 16))
    for g_, m_, c_, b in cases:
        full = oracle.render(g_, m_, c_)
        binned = oracle.render(g_, m_, c_, bin=b)
        for k in ("image", "depth", "depth01", "T_f", "n_contrib", "n_cand", "n_iter", "n_near", "tie", "gmargin"):
            np.testing.assert_array_equal(binned[k], full[k], err_msg=k)
        # a margin beyond the widened boxes (4 near_rel) may come from a Gaussian the bins leave out
        cap = 4 * oracle.NEAR
        np.testing.assert_array_equal(np.minimum(binned["margin"], cap), np.minimum(full["margin"], cap))
        pix = np.flatnonzero(full["n_near"].reshape(-1) > 0)[:20]
        if pix.size:
            a, bb = oracle.branches(g_, m_, c_, pix), oracle.branches(g_, m_, c_, pix, bin=b)
            np.testing.assert_array_equal(a["image"], bb["image"])
        G = rng.standard_normal((3, c_.height, c_.width))
        Gz = rng.standard_normal((c_.height, c_.width))
        ga = oracle.backward(g_, m_, c_, G, Gz, bin=b)
        gc = oracle.backward(g_, m_, c_, G, Gz)
        # the same per-pixel terms, summed over threads in another order
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "medium"):
            np.testing.assert_allclose(ga[k], gc[k], rtol=1e-12, atol=1e-12 * np.abs(gc[k]).max(), err_msg=k)
        assert np.abs(ga["means"]).sum() > 0
