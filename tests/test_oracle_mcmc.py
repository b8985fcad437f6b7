"""Pins of the MCMC densification oracle (Sec. IV-D adopts the sampling
form of 3DGS-MCMC; the relocation and the position noise), CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import mcmc as MC


def _logit(p):
    return math.log(p / (1.0 - p))


@pytest.mark.parametrize("o,N", [(0.9, 2), (0.3, 5), (0.05, 17), (0.999, 51), (0.5, 1)])
def test_shared_opacity_composites_back_to_the_original(o, N):
    o_new, f = MC.shared_opacity_scale(o, N)
    assert abs((1.0 - (1.0 - o_new) ** N) - o) < 1e-14
    if N == 1:
        assert o_new == pytest.approx(o, abs=1e-15) and f == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("o,N", [(0.9, 2), (0.3, 5), (0.05, 17), (0.7, 30)])
def test_scale_rule_keeps_the_line_integral(o, N):
    """The composite of N copies, 1 - (1 - o' e^{-x^2/2s'^2})^N, integrates
    along a line to the original o e^{-x^2/2s^2}: checked by quadrature."""
    s = 0.37
    o_new, f = MC.shared_opacity_scale(o, N)
    sn = f * s
    comp, _ = integrate.quad(lambda x: 1.0 - (1.0 - o_new * math.exp(-x * x / (2 * sn * sn))) ** N, -np.inf, np.inf,
                             epsabs=1e-13, epsrel=1e-12)
    assert comp == pytest.approx(o * s * math.sqrt(2 * math.pi), rel=1e-9)


def test_z_factor_hand_worked():
    o = 0.4
    assert MC.z_factor(1, o) == pytest.approx(o, abs=1e-16)
    assert MC.z_factor(2, o) == pytest.approx(2 * o - o * o / math.sqrt(2), abs=1e-15)
    assert MC.z_factor(3, o) == pytest.approx(3 * o - 3 * o * o / math.sqrt(2) + o ** 3 / math.sqrt(3), abs=1e-15)


def test_sources_follow_the_running_sum():
    logits = [_logit(0.5), _logit(0.001), _logit(0.25), _logit(0.002), _logit(0.25)]
    # live weights 0.5, 0, 0.25, 0, 0.25 -> running sum 0.5, 0.5, 0.75, 0.75, 1.0
    u = [0.0, 0.5, 0.0, 0.76, 0.0]
    dead, src = MC.sources(logits, u)
    assert dead.tolist() == [False, True, False, True, False]
    # dead 1: 0.5 * 1.0 = 0.5 -> first C > 0.5 is index 2; dead 3: 0.76 -> index 4
    assert src.tolist() == [-1, 2, -1, 4, -1]


def test_sampling_frequencies_are_proportional_to_opacity():
    """A grid of uniforms over many dead Gaussians lands on each live one in
    proportion to its opacity (exactly, for the grid)."""
    live_o = [0.8, 0.1, 0.4, 0.7]
    n_dead = 2000
    logits = np.array([_logit(p) for p in live_o] + [_logit(1e-4)] * n_dead)
    u = np.zeros(len(logits))
    u[len(live_o):] = (np.arange(n_dead) + 0.5) / n_dead
    dead, src = MC.sources(logits, u)
    counts = np.bincount(src[dead], minlength=len(live_o))[:len(live_o)]
    expect = np.array(live_o) / sum(live_o) * n_dead
    assert np.abs(counts - expect).max() <= 1.0


def test_relocate_copies_resets_and_leaves_the_rest():
    rng = np.random.default_rng(3)
    n, K = 12, 4
    logits = rng.normal(1.0, 1.0, n)
    logits[[2, 7, 9]] = _logit(0.003)
    p = {"means": rng.normal(0, 1, (n, 3)), "log_scales": rng.normal(-3, 0.4, (n, 3)),
         "quats": rng.normal(0, 1, (n, 4)), "opacity_logits": logits, "sh": rng.normal(0, 0.5, (n, K, 3))}
    m = {k: np.ones_like(v) for k, v in p.items()}
    v = {k: 2 * np.ones_like(x) for k, x in p.items()}
    u = rng.uniform(0, 1, n)
    P, M, V, n_dead = MC.relocate(p, m, v, u)
    assert n_dead == 3
    _, src = MC.sources(logits, u)
    touched = set(src[src >= 0].tolist()) | {2, 7, 9}
    for g in range(n):
        if g in touched:
            assert all((M[k][g] == 0).all() and (V[k][g] == 0).all() for k in M)
        else:
            for k in p:
                np.testing.assert_array_equal(P[k][g], p[k][g])
            assert all((M[k][g] == 1).all() for k in M)
    counts = np.bincount(src[src >= 0], minlength=n)
    for g in np.flatnonzero(counts):
        N = counts[g] + 1
        o = 1 / (1 + math.exp(-logits[g]))
        o_new, f = MC.shared_opacity_scale(o, N)
        assert 1 / (1 + math.exp(-P["opacity_logits"][g])) == pytest.approx(o_new, rel=1e-12)
        np.testing.assert_allclose(P["log_scales"][g], p["log_scales"][g] + math.log(f), rtol=1e-13)
    for d in (2, 7, 9):
        for k in p:
            np.testing.assert_array_equal(P[k][d], P[k][src[d]])


def test_noise_hand_worked():
    """Identity rotation, scales (a, b, c), eta = e_x: the mean moves by
    lambda lr gate a^2 along x, with gate = sigmoid(-k (o - t)) = 1/2 at o = t."""
    a, b, c = 0.2, 0.1, 0.05
    ls = np.log([[a, b, c]])
    mu = MC.noise(np.zeros((1, 3)), ls, np.array([[1.0, 0, 0, 0]]), [_logit(MC.NOISE_T)], np.array([[1.0, 0, 0]]),
                  lr=1e-6, lambda_noise=1e5)
    np.testing.assert_allclose(mu[0], [1e5 * 1e-6 * 0.5 * a * a, 0, 0], rtol=1e-12, atol=1e-18)
    # an opaque Gaussian barely moves: gate = sigmoid(-100 (0.9 - 0.005))
    mu2 = MC.noise(np.zeros((1, 3)), ls, np.array([[1.0, 0, 0, 0]]), [_logit(0.9)], np.array([[1.0, 0, 0]]),
                   lr=1e-6, lambda_noise=1e5)
    assert abs(mu2[0, 0]) < 1e-40
