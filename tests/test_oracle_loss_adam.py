"""Pins of the loss and Adam oracles."""
import numpy as np
import torch

from oracle import adam as oadam
from oracle import loss as oloss


def test_ssim_of_identical_images_is_one():
    x = np.random.default_rng(0).uniform(0, 1, (3, 20, 27))
    assert abs(oloss.ssim(x, x) - 1.0) < 1e-12


def test_ssim_interior_of_constant_images_closed_form():
    """Constant images a and b: away from the zero-padded border the local
    means are a, b and the variances vanish, so SSIM = (2ab + C1)/(a^2 + b^2 + C1)."""
    a, b = 0.3, 0.7
    x = torch.full((1, 30, 30), a, dtype=torch.float64)
    y = torch.full((1, 30, 30), b, dtype=torch.float64)
    s = oloss.ssim_map(x, y)[0, 5:-5, 5:-5]
    expect = (2 * a * b + oloss.C1) / (a * a + b * b + oloss.C1)
    assert torch.allclose(s, torch.full_like(s, expect), atol=1e-12)


def test_window_is_normalised_gaussian():
    w = oloss.window()
    assert abs(float(w.sum()) - 1) < 1e-15
    g = w[5] / w[5, 5]
    assert abs(float(g[6]) - np.exp(-1 / (2 * 1.5 ** 2))) < 1e-14


def test_l1_gradient_is_sign_over_count_when_lambda_zero():
    rng = np.random.default_rng(1)
    x, y = rng.uniform(0, 1, (3, 8, 9)), rng.uniform(0, 1, (3, 8, 9))
    loss, g = oloss.loss_and_grad(x, y, lam=0.0)
    assert abs(loss - np.abs(x - y).mean()) < 1e-15
    np.testing.assert_allclose(g, np.sign(x - y) / x.size, atol=1e-16)


def test_loss_gradient_central_differences():
    rng = np.random.default_rng(2)
    x, y = rng.uniform(0, 1, (3, 14, 17)), rng.uniform(0, 1, (3, 14, 17))
    _, g = oloss.loss_and_grad(x, y, lam=0.2)
    for _ in range(12):
        idx = tuple(int(rng.integers(0, s)) for s in x.shape)
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oloss.loss_and_grad(xp, y)[0] - oloss.loss_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8 + 1e-5 * abs(fd)


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(4)]
    tp = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step, g in enumerate(grads, start=1):
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = oadam.adam_step(p, g, m, v, step, lr=0.01)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)
