"""The oracle's analytic FP64 adjoint against FP64 central finite differences.

L = <G, image> + <Gz, depth> + <G01, depth01> with random upstream G. Each
probed parameter x is moved by h = 1e-6 max(1, |x|); the scene is chosen so
that no pixel is within 1e-4 of a discrete decision (3-sigma cut, alpha skip,
transmittance stop) or of a clamp, so every FD difference stays on one smooth
branch of the rendering function.
"""
import numpy as np
import pytest

import oracle
from paper_2411_19588_b300 import scenes


def _scene(seed, deg=3, n=60, W=48, H=36):
    rng = np.random.default_rng(seed)
    cam = scenes.look_at([0.2, -0.1, -0.3], [0.0, 0.05, 3.0], W, H, 45.0, 45.0)
    means = np.c_[rng.uniform(-0.9, 0.9, (n, 2)), rng.uniform(1.5, 5.0, n)]
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.1, (n, K, 3))
    sh[:, 0, :] = (rng.uniform(0.2, 0.8, (n, 3)) - 0.5) / 0.28209479177387814
    g = scenes.Gaussians(*(np.ascontiguousarray(a, np.float32) for a in (
        means, rng.normal(-1.9, 0.3, (n, 3)), rng.standard_normal((n, 4)), rng.normal(0.3, 1.0, n), sh)), deg)
    med = scenes.random_medium(rng)
    return g, med, cam


def _clean_scene(deg):
    for seed in range(60):
        g, med, cam = _scene(seed, deg)
        r = oracle.render(g, med, cam)
        if r["margin"].min() > 1e-4 and r["gmargin"].min() > 1e-3 and r["tie"].sum() == 0:
            return g, med, cam, r
    pytest.fail("no decision-clean scene found")


def _loss(g, med_arr, cam, G, Gz, G01):
    r = oracle.render(g, med_arr, cam)
    return float((G * r["image"]).sum() + (Gz * r["depth"]).sum() + (G01 * r["depth01"]).sum())


def _as64(g):
    return scenes.Gaussians(*(np.asarray(a, np.float64).copy() for a in (g.means, g.log_scales, g.quats,
                                                                          g.opacity_logits, g.sh)), g.sh_degree)


@pytest.mark.parametrize("deg", [0, 3])
def test_oracle_gradients_match_central_differences(deg):
    g32, med, cam, r = _clean_scene(deg)
    g = _as64(g32)
    med_arr = med.as_array().astype(np.float64)
    rng = np.random.default_rng(100 + deg)
    G = rng.standard_normal((3, cam.height, cam.width))
    Gz = rng.standard_normal((cam.height, cam.width)) * 0.05
    G01 = rng.standard_normal((cam.height, cam.width)) * 0.3
    grads = oracle.backward(g, med_arr, cam, G, Gz, G01)

    contributing = np.nonzero(np.abs(grads["proj"]).sum(1) > 0)[0]
    assert contributing.size >= 10
    probes = [("medium", (j,)) for j in range(9)]
    for i in rng.choice(contributing, 8, replace=False):
        probes += [("means", (i, k)) for k in range(3)]
        probes += [("log_scales", (i, k)) for k in range(3)]
        probes += [("quats", (i, k)) for k in range(4)]
        probes += [("opacity_logits", (i,))]
        probes += [("sh", (i, k, c)) for k, c in [(0, 0), (0, 2)] + ([(1, 1), (5, 0), (11, 2), (15, 1)] if deg == 3 else [])]

    worst = 0.0
    for name, idx in probes:
        def L_at(delta):
            gg = _as64(g)
            m = med_arr.copy()
            if name == "medium":
                m[idx] += delta
            else:
                getattr(gg, name)[idx] += delta
            return _loss(gg, m, cam, G, Gz, G01)

        x = med_arr[idx] if name == "medium" else getattr(g, name)[idx]
        h = 1e-6 * max(1.0, abs(float(x)))
        fd = (L_at(h) - L_at(-h)) / (2 * h)
        an = float(grads[name][idx])
        err = abs(fd - an) / max(1e-3, abs(fd), abs(an))
        worst = max(worst, err)
        assert err < 2e-5, (name, idx, fd, an)
    assert worst < 2e-5
    # the scene overlaps enough to exercise the transmittance terms
    assert r["n_contrib"].mean() > 3 and r["n_contrib"].max() >= 10


def test_noncontributing_gaussians_get_zero_gradient():
    g, med, cam, _ = _clean_scene(0)
    g = _as64(g)
    # push one Gaussian behind the camera
    g.means[0] = [0.0, 0.0, -3.0]
    G = np.ones((3, cam.height, cam.width))
    grads = oracle.backward(g, med.as_array(), cam, G)
    assert np.all(grads["means"][0] == 0) and np.all(grads["sh"][0] == 0) and grads["opacity_logits"][0] == 0
