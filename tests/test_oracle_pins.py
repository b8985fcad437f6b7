"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with an
independent statement (a plain Eq. 1 composite, a closed form, a library
routine, an algebraic identity or brute force).
"""
import math

import numpy as np
import pytest
import scipy.special
from scipy.spatial.transform import Rotation

import oracle
from paper_2411_19588_b300 import scenes


def _gauss(means, log_scales, quats, logits, sh, deg):
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return scenes.Gaussians(f(means), f(log_scales), f(quats), f(logits), f(sh), deg)


def _cam(W=64, H=48, f=60.0, w2c=None, z_far=20.0):
    if w2c is None:
        w2c = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    return scenes.Camera(W, H, f, f, W / 2.0, H / 2.0, w2c, 0.2, z_far)


def _medium(bd, bb, binf):
    return scenes.Medium(np.asarray(bd, np.float32), np.asarray(bb, np.float32), np.asarray(binf, np.float32))


def plain_composite(proj, px, py):
    """Eq. 1 written out in the test: sort the Gaussians whose 3-sigma
    ellipse holds the pixel by (depth, index), alpha = min(0.99, opac*e^{-q/2}),
    skip alpha < 1/255, stop before T would drop below 1e-4."""
    vis = proj["vis"] > 0
    dx, dy = px - proj["x"], py - proj["y"]
    q = proj["KA"] * dx * dx + 2 * proj["KB"] * dx * dy + proj["KC"] * dy * dy
    idx = np.nonzero(vis & (q <= 9.0))[0]
    idx = idx[np.lexsort((idx, proj["d"][idx]))]
    C, T, D, A = np.zeros(3), 1.0, 0.0, 0.0
    col = np.stack([proj["col_r"], proj["col_g"], proj["col_b"]], 1)
    for i in idx:
        a = min(0.99, proj["opac"][i] * math.exp(-0.5 * q[i]))
        if a < 1 / 255:
            continue
        if T * (1 - a) < 1e-4:
            break
        C += col[i] * a * T
        D += proj["d"][i] * a * T
        A += a * T
        T *= 1 - a
    return C, T, D, A


def test_beta_zero_is_plain_compositing():
    """With beta_D = beta_B = 0 the water terms vanish (Eq. 5 -> Eq. 1),
    whatever B_inf is."""
    g, _, cam = scenes.tiny_scene(0)
    med = _medium([0, 0, 0], [0, 0, 0], [0.3, 0.6, 0.9])
    r = oracle.render(g, med, cam)
    proj = oracle.project(g, med, cam)
    rng = np.random.default_rng(1)
    for p in rng.choice(cam.width * cam.height, 300, replace=False):
        iy, ix = divmod(int(p), cam.width)
        C, T, D, A = plain_composite(proj, ix + 0.5, iy + 0.5)
        np.testing.assert_allclose(r["image"][:, iy, ix], C, rtol=0, atol=1e-12)
        assert abs(r["T_f"][iy, ix] - T) < 1e-12
        z = D / A if A > 0 else cam.z_far
        assert abs(r["depth"][iy, ix] - z) < 1e-9


def test_empty_scene_is_pure_backscatter():
    """No Gaussians (or all behind the camera): C = B_inf (1 - e^{-beta_B z_far}),
    z = z_far, T = 1."""
    med = _medium([0.4, 0.2, 0.1], [0.3, 0.25, 0.2], [0.05, 0.2, 0.3])
    cam = _cam()
    expect = np.array([0.05, 0.2, 0.3]) * (1 - np.exp(-np.array([0.3, 0.25, 0.2]) * cam.z_far))
    empty = _gauss(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 4)), np.zeros(0), np.zeros((0, 1, 3)), 0)
    rng = np.random.default_rng(2)
    behind = _gauss(np.c_[rng.uniform(-1, 1, (20, 2)), rng.uniform(-5, 0.1, 20)], np.full((20, 3), -1.0),
                    np.tile([1.0, 0, 0, 0], (20, 1)), np.full(20, 3.0), np.zeros((20, 1, 3)), 0)
    for g in (empty, behind):
        r = oracle.render(g, med, cam)
        np.testing.assert_allclose(r["image"], np.broadcast_to(expect[:, None, None], r["image"].shape), atol=1e-14)
        np.testing.assert_allclose(r["depth"], cam.z_far)
        np.testing.assert_allclose(r["T_f"], 1.0)


@pytest.mark.parametrize("logit", [-1.0, 0.5, 8.0])
def test_single_gaussian_centre_closed_form(logit):
    """A single Gaussian whose projected centre is a pixel centre: q = 0 there, so
    alpha = min(0.99, sigmoid(o)) and
    C = c alpha e^{-beta_D d} + B_inf (1 - e^{-beta_B d}) + (1 - alpha) B_inf (e^{-beta_B d} - e^{-beta_B z_far}),
    z = d, z01 = 2/(1+e^{-0.1 d}) - 1."""
    cam = _cam(W=64, H=48, f=60.0)
    ix, iy, d = 40, 17, 4.25
    mx = (ix + 0.5 - cam.cx) * d / cam.fx
    my = (iy + 0.5 - cam.cy) * d / cam.fy
    rgb = np.array([0.8, 0.5, 0.2])
    sh0 = (rgb - 0.5) / (0.5 / math.sqrt(math.pi))
    g = _gauss([[mx, my, d]], [[-2.0, -2.5, -1.8]], [[0.9, 0.1, -0.3, 0.2]], [logit], sh0[None, None, :], 0)
    bd, bb, binf = np.array([0.4, 0.2, 0.1]), np.array([0.3, 0.25, 0.2]), np.array([0.05, 0.2, 0.3])
    med = _medium(bd, bb, binf)
    r = oracle.render(g, med, cam)
    # the float32 storage of the inputs moves the centre by ~1e-7 px
    gf = g.means.astype(np.float64)[0]
    assert abs(cam.fx * gf[0] / gf[2] + cam.cx - (ix + 0.5)) < 1e-5
    dd = float(gf[2])
    alpha = min(0.99, 1 / (1 + math.exp(-np.float64(np.float32(logit)))))
    rgbf = 0.5 + g.sh.astype(np.float64)[0, 0] * 0.5 / math.sqrt(math.pi)
    f64 = lambda v: v.astype(np.float32).astype(np.float64)
    a, b, bfar = np.exp(-f64(bd) * dd), np.exp(-f64(bb) * dd), np.exp(-f64(bb) * cam.z_far)
    binf32 = f64(binf)
    expect = rgbf * alpha * a + binf32 * (1 - b) + (1 - alpha) * binf32 * (b - bfar)
    np.testing.assert_allclose(r["image"][:, iy, ix], expect, rtol=0, atol=1e-9)
    assert abs(r["depth"][iy, ix] - dd) < 1e-12
    assert abs(r["depth01"][iy, ix] - (2 / (1 + math.exp(-0.1 * dd)) - 1)) < 1e-12


def test_opaque_stack_approaches_eq4():
    """Stacked opaque Gaussians at (nearly) one depth d: the pixel saturates and
    C -> c e^{-beta_D d} + B_inf (1 - e^{-beta_B d}), the single-surface
    Sea-thru formation (Eq. 3 / Eq. 4), within the 1e-4 transmittance floor."""
    cam = _cam(W=32, H=32, f=40.0)
    ix, iy, d = 15, 9, 3.0
    n = 6
    ds = d + 1e-7 * np.arange(n)
    mx = (ix + 0.5 - cam.cx) * ds / cam.fx
    my = (iy + 0.5 - cam.cy) * ds / cam.fy
    rgb = np.array([0.7, 0.3, 0.9])
    sh0 = np.tile((rgb - 0.5) / (0.5 / math.sqrt(math.pi)), (n, 1))[:, None, :]
    g = _gauss(np.c_[mx, my, ds], np.full((n, 3), -2.0), np.tile([1.0, 0, 0, 0], (n, 1)), np.full(n, 30.0), sh0, 0)
    bd, bb, binf = np.array([0.35, 0.15, 0.05]), np.array([0.4, 0.3, 0.2]), np.array([0.1, 0.3, 0.5])
    r = oracle.render(g, _medium(bd, bb, binf), cam)
    eq4 = rgb * np.exp(-bd * d) + binf * (1 - np.exp(-bb * d))
    np.testing.assert_allclose(r["image"][:, iy, ix], eq4, rtol=0, atol=2e-4 * 1.5)
    assert r["n_contrib"][iy, ix] == 2  # 0.99 then 0.0099; the third would take T below 1e-4


def _random_list(rng, m):
    alpha = rng.uniform(0.01, 0.9, m)
    col = rng.uniform(0, 1, (m, 3))
    d = np.sort(rng.uniform(0.5, 15, m))
    med = np.r_[rng.uniform(0.05, 0.6, 6), rng.uniform(0.05, 0.4, 3)]
    return alpha, col, d, med


def test_zero_alpha_insertions_are_invisible():
    """Splitting a water segment with an alpha = 0 Gaussian at any depth
    leaves colour, transmittance and depth sums unchanged."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        m = int(rng.integers(0, 12))
        alpha, col, d, med = _random_list(rng, m)
        base = oracle.composite(alpha, col, d, med, 20.0)
        k = int(rng.integers(1, 5))
        d_new = rng.uniform(0.3, 19.9, k)
        A = np.r_[alpha, np.zeros(k)]
        Cc = np.r_[col, rng.uniform(0, 1, (k, 3))]
        D = np.r_[d, d_new]
        o = np.argsort(D, kind="stable")
        ins = oracle.composite(A[o], Cc[o], D[o], med, 20.0)
        np.testing.assert_allclose(ins[0], base[0], atol=1e-13)
        assert abs(ins[1] - base[1]) < 1e-14 and abs(ins[2] - base[2]) < 1e-12 and abs(ins[3] - base[3]) < 1e-13


def test_segment_sum_telescopes():
    """sum_i c a alpha T + B sum_segments T (b_prev - b) ==
    sum_i alpha T (c a - B b) + B (1 - T_final b_far): the per-Gaussian
    effective-colour form, derived by summation by parts."""
    rng = np.random.default_rng(4)
    for _ in range(30):
        m = int(rng.integers(0, 15))
        alpha, col, d, med = _random_list(rng, m)
        zfar = 20.0
        rgb, Tf, _, _ = oracle.composite(alpha, col, d, med, zfar)
        T = np.concatenate([[1.0], np.cumprod(1 - alpha)])[:m]
        a = np.exp(-np.outer(d, med[0:3]))
        b = np.exp(-np.outer(d, med[3:6]))
        tele = ((alpha * T)[:, None] * (col * a - med[6:9] * b)).sum(0) + med[6:9] * (1 - np.prod(1 - alpha) * np.exp(-med[3:6] * zfar))
        np.testing.assert_allclose(rgb, tele, atol=1e-13)
        assert abs(Tf - np.prod(1 - alpha)) < 1e-15


def test_input_order_does_not_matter():
    """Compositing sorts by depth: permuting the Gaussian buffers (distinct
    depths) leaves the image unchanged."""
    g, m, cam = scenes.tiny_scene(0)
    r0 = oracle.render(g, m, cam)
    perm = np.random.default_rng(5).permutation(g.n)
    r1 = oracle.render(g.subset(perm), m, cam)
    np.testing.assert_allclose(r1["image"], r0["image"], atol=1e-13)
    np.testing.assert_allclose(r1["depth"], r0["depth"], atol=1e-11)


def test_degree0_colour_is_drawn_rgb():
    g, m, cam = scenes.tiny_scene(0)
    proj = oracle.project(g, m, cam)
    rgb = 0.5 + g.sh[:, 0, :].astype(np.float64) * 0.5 / math.sqrt(math.pi)
    vis = proj["vis"] > 0
    got = np.stack([proj["col_r"], proj["col_g"], proj["col_b"]], 1)
    np.testing.assert_allclose(got[vis], np.maximum(rgb[vis], 0), atol=1e-12)
    # the generator draws RGB in [0, 1]
    assert rgb.min() > -1e-6 and rgb.max() < 1 + 1e-6


def _sphere_quadrature(nt=24, nphi=48):
    ct, w = np.polynomial.legendre.leggauss(nt)
    phi = np.arange(nphi) * 2 * np.pi / nphi
    CT, PH = np.meshgrid(ct, phi, indexing="ij")
    st = np.sqrt(1 - CT ** 2)
    dirs = np.stack([st * np.cos(PH), st * np.sin(PH), CT], -1).reshape(-1, 3)
    weights = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return dirs, weights


def test_sh_basis_orthonormal():
    """Real SH up to degree 3 are orthonormal on the sphere (exact quadrature)."""
    dirs, w = _sphere_quadrature()
    Y = np.stack([oracle.sh_basis(3, d) for d in dirs])
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_basis_matches_scipy():
    """Real form of scipy's complex spherical harmonics: m>0 -> sqrt2 (-1)^m Re Y_l^m,
    m<0 -> sqrt2 (-1)^m Im Y_l^|m|, m=0 -> Y_l^0."""
    rng = np.random.default_rng(6)
    for _ in range(25):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        theta, phi = math.acos(v[2]), math.atan2(v[1], v[0])
        Y = oracle.sh_basis(3, v)
        for l in range(4):
            for m in range(-l, l + 1):
                c = scipy.special.sph_harm_y(l, abs(m), theta, phi)
                ref = c.real if m == 0 else math.sqrt(2) * (-1) ** m * (c.real if m > 0 else c.imag)
                assert abs(Y[l * l + l + m] - ref) < 1e-12, (l, m)


def test_projection_matches_fd_jacobian_and_scipy_rotation():
    """Sigma2 - 0.3 I = J W Sigma3 W^T J^T with Sigma3 from scipy's quaternion
    rotation and J the central-difference Jacobian of the pinhole map; the
    centre is the pinhole image of the mean; the conic is the inverse."""
    rng = np.random.default_rng(7)
    cam = scenes.look_at([0.3, -0.2, -0.5], [0.1, 0.05, 4.0], 96, 64, 80.0, 80.0)
    n = 40
    means = np.c_[rng.uniform(-0.8, 0.8, (n, 2)), rng.uniform(2, 6, n)]
    g = _gauss(means, rng.normal(-2, 0.5, (n, 3)), rng.standard_normal((n, 4)), rng.normal(0, 1, n),
               rng.normal(0, 0.1, (n, 4, 3)), 1)
    proj = oracle.project(g, _medium([0.1] * 3, [0.1] * 3, [0.1] * 3), cam)
    W = cam.world_to_cam[:, :3]
    t0 = cam.world_to_cam[:, 3]
    pin = lambda t: np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
    for i in range(n):
        mu = g.means[i].astype(np.float64)
        t = W @ mu + t0
        assert proj["vis"][i] == 1
        np.testing.assert_allclose([proj["x"][i], proj["y"][i]], pin(t), rtol=1e-13)
        J = np.zeros((2, 3))
        for k in range(3):
            h = np.zeros(3)
            h[k] = 1e-6
            J[:, k] = (pin(t + h) - pin(t - h)) / 2e-6
        q = g.quats[i].astype(np.float64)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = np.diag(np.exp(2 * g.log_scales[i].astype(np.float64)))
        S2 = J @ W @ Rq @ S @ Rq.T @ W.T @ J.T
        got = np.array([[proj["SA"][i] - 0.3, proj["SB"][i]], [proj["SB"][i], proj["SC"][i] - 0.3]])
        np.testing.assert_allclose(got, S2, rtol=1e-6, atol=1e-8 * np.abs(S2).max())
        K = np.linalg.inv(got + 0.3 * np.eye(2))
        np.testing.assert_allclose([proj["KA"][i], proj["KB"][i], proj["KC"][i]], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-9)


def test_isotropic_on_axis_conic():
    """Isotropic Gaussian (scale s) on the optical axis at depth z:
    conic = 1 / (s^2 f^2 / z^2 + 0.3) * I."""
    cam = _cam(W=64, H=64, f=70.0)
    for s, z in [(0.05, 2.0), (0.01, 7.5), (0.2, 12.0)]:
        g = _gauss([[0, 0, z]], [[math.log(s)] * 3], [[0.3, -0.5, 0.2, 0.7]], [0.0], np.zeros((1, 1, 3)), 0)
        proj = oracle.project(g, _medium([0] * 3, [0] * 3, [0] * 3), cam)
        sf = np.float64(np.float32(math.log(s)))
        k = 1.0 / (math.exp(2 * sf) * cam.fx ** 2 / z ** 2 + 0.3)
        np.testing.assert_allclose([proj["KA"][0], proj["KB"][0], proj["KC"][0]], [k, 0, k], rtol=1e-12, atol=1e-14)


def test_pixel_subset_matches_full_render():
    g, m, cam = scenes.tiny_scene(0)
    full = oracle.render(g, m, cam)
    pix = np.random.default_rng(8).choice(cam.width * cam.height, 200, replace=False)
    sub = oracle.render(g, m, cam, pix=pix)
    iy, ix = np.divmod(pix, cam.width)
    np.testing.assert_array_equal(sub["image"], full["image"][:, iy, ix])
    np.testing.assert_array_equal(sub["depth"], full["depth"][iy, ix])


def test_tiny_scene_margins_are_rare():
    """Pixels within 1e-5 (relative) of a discrete decision are rare; the GPU
    parity tests exclude and count them."""
    g, m, cam = scenes.tiny_scene(0)
    r = oracle.render(g, m, cam)
    assert (r["margin"] < 1e-5).mean() < 1e-3
    assert r["tie"].sum() == 0
