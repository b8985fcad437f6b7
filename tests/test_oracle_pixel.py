"""Pins for the pixel-mode oracle (Eq. 5 with the Eq. 6 depth): closed forms,
limits, the paper's appendix derivatives, and FP64 central differences of
the whole pixel-mode loss (including the dependence of z on the Gaussians)."""
import math

import numpy as np
import pytest

import oracle
from oracle import pixel as P
from paper_2411_19588_b300 import scenes

from test_oracle_pins import _cam, _gauss, _medium
from test_oracle_grad_fd import _as64, _clean_scene


def test_empty_scene_is_pure_backscatter():
    med = _medium([0.4, 0.2, 0.1], [0.3, 0.25, 0.2], [0.05, 0.2, 0.3])
    cam = _cam()
    empty = _gauss(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), np.zeros(0), np.zeros((0, 1, 3)), 0)
    r = P.render(empty, med, cam)
    expect = np.array([0.05, 0.2, 0.3]) * (1 - np.exp(-np.array([0.3, 0.25, 0.2]) * cam.z_far))
    np.testing.assert_allclose(r["image"], np.broadcast_to(expect[:, None, None], r["image"].shape), atol=1e-14)


@pytest.mark.parametrize("logit", [-1.0, 0.5, 8.0])
def test_single_gaussian_centre_closed_form(logit):
    """Eq. 5 at the centre pixel of a lone Gaussian: J = c alpha, z = d, so
    C = c alpha e^{-beta_D d} + B_inf (1 - e^{-beta_B d}) (no water behind it,
    unlike the segment model)."""
    cam = _cam(W=64, H=48, f=60.0)
    ix, iy, d = 40, 17, 4.25
    mx, my = (ix + 0.5 - cam.cx) * d / cam.fx, (iy + 0.5 - cam.cy) * d / cam.fy
    rgb = np.array([0.8, 0.5, 0.2])
    sh0 = (rgb - 0.5) / (0.5 / math.sqrt(math.pi))
    g = _gauss([[mx, my, d]], [[-2.0, -2.5, -1.8]], [[0.9, 0.1, -0.3, 0.2]], [logit], sh0[None, None, :], 0)
    bd, bb, binf = np.array([0.4, 0.2, 0.1]), np.array([0.3, 0.25, 0.2]), np.array([0.05, 0.2, 0.3])
    r = P.render(g, _medium(bd, bb, binf), cam)
    f64 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    dd = float(g.means.astype(np.float64)[0, 2])
    alpha = min(0.99, 1 / (1 + math.exp(-np.float64(np.float32(logit)))))
    rgbf = 0.5 + g.sh.astype(np.float64)[0, 0] * 0.5 / math.sqrt(math.pi)
    expect = rgbf * alpha * np.exp(-f64(bd) * dd) + f64(binf) * (1 - np.exp(-f64(bb) * dd))
    np.testing.assert_allclose(r["image"][:, iy, ix], expect, rtol=0, atol=1e-9)


def test_opaque_surface_reaches_eq4_and_agrees_with_segment_model():
    """A saturated pixel (opaque stack at one depth d) gives the single-surface
    formation of Eq. 3/4 in both models: c e^{-beta_D d} + B_inf (1 - e^{-beta_B d})."""
    cam = _cam(W=32, H=32, f=40.0)
    ix, iy, d, n = 15, 9, 3.0, 6
    ds = d + 1e-7 * np.arange(n)
    mx, my = (ix + 0.5 - cam.cx) * ds / cam.fx, (iy + 0.5 - cam.cy) * ds / cam.fy
    rgb = np.array([0.3, 0.6, 0.9])
    sh0 = np.tile((rgb - 0.5) / (0.5 / math.sqrt(math.pi)), (n, 1))[:, None, :]
    g = _gauss(np.c_[mx, my, ds], np.full((n, 3), -1.0), np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, 12.0), sh0, 0)
    med = _medium([0.4, 0.2, 0.1], [0.3, 0.25, 0.2], [0.05, 0.2, 0.3])
    rp = P.render(g, med, cam)
    rs = oracle.render(g, med, cam)
    m = med.as_array().astype(np.float64)
    expect = rgb * np.exp(-m[0:3] * d) + m[6:9] * (1 - np.exp(-m[3:6] * d))
    np.testing.assert_allclose(rp["image"][:, iy, ix], expect, atol=2e-4)
    np.testing.assert_allclose(rp["image"][:, iy, ix], rs["image"][:, iy, ix], atol=3e-4)


def test_zero_medium_is_plain_compositing():
    g, _, cam = scenes.tiny_scene(0)
    z = _medium([0, 0, 0], [0, 0, 0], [0, 0, 0])
    np.testing.assert_array_equal(P.render(g, z, cam)["image"], oracle.render(g, z, cam)["image"])


def test_medium_gradients_match_the_paper_appendix():
    """The appendix's partial derivatives of Eq. 5 at fixed z: dL/dB_inf =
    G (1 - e^{-beta_B z}) as printed; dL/dbeta_D and dL/dbeta_B as printed
    but with the factor z that differentiating e^{-beta z} brings (the printed
    forms omit it) and without the stray lambda_est."""
    g, med, cam = scenes.tiny_scene(0)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, cam.height, cam.width))
    res = P.backward(g, med, cam, G)
    r = P.render(g, med, cam)
    m = med.as_array().astype(np.float64)
    z, J = r["depth"], r["J"]
    a = np.exp(-m[0:3, None, None] * z)
    b = np.exp(-m[3:6, None, None] * z)
    np.testing.assert_allclose(res["medium"][6:9], (G * (1 - b)).sum((1, 2)), rtol=1e-12)
    np.testing.assert_allclose(res["medium"][0:3], (-(J * a) * G * z).sum((1, 2)), rtol=1e-12)
    np.testing.assert_allclose(res["medium"][3:6], (G * m[6:9, None, None] * b * z).sum((1, 2)), rtol=1e-12)


def test_pixel_mode_gradients_match_central_differences():
    g32, med, cam, _ = _clean_scene(3)
    g = _as64(g32)
    m0 = med.as_array().astype(np.float64)
    rng = np.random.default_rng(7)
    G = rng.standard_normal((3, cam.height, cam.width))
    Gz = rng.standard_normal((cam.height, cam.width)) * 0.05
    grads = P.backward(g, m0, cam, G, Gz)

    def loss(gg, m):
        r = P.render(gg, m, cam)
        return float((G * r["image"]).sum() + (Gz * r["depth"]).sum())

    contributing = np.nonzero(np.abs(grads["means"]).sum(1) > 0)[0]
    probes = [("medium", (j,)) for j in range(9)]
    for i in rng.choice(contributing, 6, replace=False):
        probes += [("means", (i, k)) for k in range(3)] + [("opacity_logits", (i,))] + [("log_scales", (i, 0))]
        probes += [("sh", (i, 0, 1))]
    for name, idx in probes:
        def L_at(delta):
            gg = _as64(g)
            m = m0.copy()
            if name == "medium":
                m[idx] += delta
            else:
                getattr(gg, name)[idx] += delta
            return loss(gg, m)
        x = m0[idx] if name == "medium" else getattr(g, name)[idx]
        h = 1e-6 * max(1.0, abs(float(x)))
        fd = (L_at(h) - L_at(-h)) / (2 * h)
        an = float(grads[name][idx])
        assert abs(fd - an) <= 2e-5 * max(1e-3, abs(fd), abs(an)), (name, idx, fd, an)
