"""Pins of the densification oracle (appendix schedule; the 3DGS procedure)."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import densify as D


def _params(n, rng, deg=1):
    k = (deg + 1) ** 2
    return {"means": rng.normal(0, 1, (n, 3)), "log_scales": rng.normal(-3, 0.5, (n, 3)),
            "quats": rng.normal(0, 1, (n, 4)), "opacity_logits": rng.normal(0, 2, n), "sh": rng.normal(0, 1, (n, k, 3))}


def test_stat_is_the_ndc_norm():
    g = np.array([[3.0, 0.0], [0.0, 2.0], [1.0, 1.0]])
    np.testing.assert_allclose(D.stat_increment(g, 200, 100), [300.0, 100.0, math.hypot(100.0, 50.0)])


def test_classify_hand_worked():
    ls = np.log(np.array([[0.01, 0.02, 0.01], [0.5, 0.1, 0.1], [0.01, 0.01, 0.01], [0.5, 0.5, 0.5], [0.3, 0.1, 0.1]]))
    logits = np.array([0.0, 0.0, 0.0, -3.0, 0.0])        # the fourth: opacity 0.047 < 0.1
    stats = np.array([[0.003, 10], [0.005, 10], [0.001, 10], [1.0, 1], [0.0, 0]])
    act = D.classify(ls, logits, stats, threshold=0.0002, min_opacity=0.1, dense=0.2)
    assert act.tolist() == [D.CLONE, D.SPLIT, D.KEEP, D.PRUNE, D.KEEP]


def test_classify_margins_and_flips():
    """Relative distances of each decision to its threshold, and the action
    when a decision is taken the other way (hand-worked)."""
    ls = np.log(np.array([[0.01, 0.02, 0.01], [0.5, 0.1, 0.1], [0.2, 0.1, 0.1]]))
    logits = np.array([0.0, math.log(0.1 / 0.9), 0.0])     # opacities 0.5, 0.1, 0.5
    stats = np.array([[0.003, 10], [0.005, 10], [0.0004, 2]])
    mg = D.decision_margins(ls, logits, stats, threshold=0.0002, min_opacity=0.1, dense=0.2)
    np.testing.assert_allclose(mg[:, 0], [4.0, 0.0, 4.0], atol=1e-15)
    np.testing.assert_allclose(mg[:, 1], [0.5, 1.5, 0.0], atol=1e-12)
    np.testing.assert_allclose(mg[:, 2], [0.9, 1.5, 0.0], atol=1e-12)
    # exactly on the thresholds: opacity 0.1 is not below 0.1, 0.0002 is selected, 0.2 is not larger than 0.2
    assert D.classify(ls, logits, stats, threshold=0.0002, min_opacity=0.1, dense=0.2).tolist() == \
        [D.CLONE, D.SPLIT, D.CLONE]
    flip = [D.SELECTED, D.LOW_OPACITY, D.LARGE]
    assert D.classify(ls, logits, stats, threshold=0.0002, min_opacity=0.1, dense=0.2, flip=flip).tolist() == \
        [D.KEEP, D.PRUNE, D.SPLIT]
    flip = [D.LOW_OPACITY | D.SELECTED, 0, D.SELECTED | D.LARGE]
    assert D.classify(ls, logits, stats, threshold=0.0002, min_opacity=0.1, dense=0.2, flip=flip).tolist() == \
        [D.PRUNE, D.SPLIT, D.KEEP]


def test_rotation_matches_scipy():
    q = np.array([0.3, -0.5, 0.2, 0.9])
    want = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x, y, z, w)
    np.testing.assert_allclose(D.rotation(q), want, atol=1e-14)


def test_apply_counts_order_moments_and_split_samples():
    rng = np.random.default_rng(0)
    p = _params(4, rng)
    m = {k: np.ones_like(v) for k, v in p.items()}
    v = {k: 2 * np.ones_like(x) for k, x in p.items()}
    act = np.array([D.KEEP, D.CLONE, D.PRUNE, D.SPLIT])
    eps = np.zeros((4, 2, 3))
    eps[3, 1] = [1.0, 0.0, 0.0]
    P, M, V = D.apply(p, m, v, act, eps)
    assert P["means"].shape == (1 + 2 + 0 + 2, 3)
    np.testing.assert_array_equal(P["means"][0], p["means"][0])
    np.testing.assert_array_equal(P["means"][1], p["means"][1])
    np.testing.assert_array_equal(P["means"][2], p["means"][1])
    assert np.all(M["sh"][0] == 1) and np.all(M["sh"][1] == 1) and np.all(M["sh"][2] == 0)
    assert np.all(V["quats"][1] == 2) and np.all(V["quats"][3:] == 0)
    # split samples: eps = 0 stays at the mean; eps = e_x moves by s_x along R's first column
    np.testing.assert_allclose(P["means"][3], p["means"][3])
    s = np.exp(p["log_scales"][3])
    np.testing.assert_allclose(P["means"][4], p["means"][3] + D.rotation(p["quats"][3])[:, 0] * s[0], rtol=1e-14)
    np.testing.assert_allclose(P["log_scales"][3:], np.broadcast_to(p["log_scales"][3] - math.log(1.6), (2, 3)))
    np.testing.assert_array_equal(P["sh"][3], p["sh"][3])


def test_split_samples_follow_the_gaussian():
    """Many split samples of one Gaussian have its covariance R S^2 R^T."""
    rng = np.random.default_rng(1)
    p = _params(1, rng)
    n = 40000
    reps = {k: np.repeat(x, n, axis=0) for k, x in p.items()}
    z = {k: np.zeros_like(x) for k, x in reps.items()}
    P, _, _ = D.apply(reps, z, z, np.full(n, D.SPLIT), rng.standard_normal((n, 2, 3)))
    R, s = D.rotation(p["quats"][0]), np.exp(p["log_scales"][0])
    cov = np.cov((P["means"] - p["means"][0]).T)
    np.testing.assert_allclose(cov, R @ np.diag(s ** 2) @ R.T, atol=0.02 * s.max() ** 2)
