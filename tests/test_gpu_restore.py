"""GPU parity of water removal (the per-pixel inverse of Eq. 5) and of the
clean render (zero medium) against the FP64 oracles."""
import numpy as np
import pytest
import torch

import oracle
from oracle import restore as RS
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes
from tests import parity, water

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -24


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    r = R.Renderer()
    yield r
    r.close()


def _tol(img, z, med, out):
    """FP32 error bound of the inverse: the clipped difference carries a few
    ulps of |I| + B_inf, scaled by a = exp(beta_D z); the product and the two
    exponentials add a few ulps of |out| (1 + beta_D z)."""
    a = np.exp(med[0:3, None, None] * z[None])
    return 8 * EPS * (a * (np.abs(img) + med[6:9, None, None]) + np.abs(out) * (1 + med[0:3, None, None] * z[None]))


@pytest.mark.parametrize("W,H", [(1920, 1280), (37, 23), (450, 301)])
def test_restore_matches_oracle(renderer, W, H):
    img, depth, med = water.view(7, W, H)
    m = med.as_array()
    out = renderer.restore(torch.from_numpy(img).cuda(), torch.from_numpy(depth).cuda(),
                           torch.from_numpy(m).cuda()).cpu().numpy()
    want = RS.restore(img, depth, m)
    err = np.abs(out - want)
    assert np.all(err <= _tol(img, depth.astype(np.float64), m.astype(np.float64), want)), err.max()
    # in place, through a misaligned view (scalar path)
    buf = torch.zeros(3 * H * W + 1, device="cuda")
    x = buf[1:].view(3, H, W)
    x.copy_(torch.from_numpy(img))
    renderer.restore(x, torch.from_numpy(depth).cuda(), torch.from_numpy(m).cuda(), out=x)
    assert np.array_equal(x.cpu().numpy(), out)


def test_clean_render_is_the_zero_medium_composite(renderer):
    g, _, cam = scenes.tiny_scene(4)
    img, depth, d01 = renderer.render_clean(R.params_to_device(g), cam)
    zero = scenes.Medium(np.zeros(3, np.float32), np.zeros(3, np.float32), np.zeros(3, np.float32))
    ora = oracle.render(g, zero, cam)
    parity.compare_forward({"image": img.cpu().numpy(), "depth": depth.cpu().numpy(), "depth01": d01.cpu().numpy()},
                           ora, label="clean")


def test_restoring_a_render_approaches_the_clean_render(renderer):
    """Rendered through water, then restored with the rendered depth and the
    same water: close to the clean render where one opaque surface fills
    the pixel (the segment model and Eq. 5 agree there)."""
    g, med, _ = scenes.patch_scene(60_000, 22, (2.0, 15.0), 480, 320, 450.0)
    cam = scenes.arc_cameras(20, 22, width=480, height=320, fx=450.0)[10]
    p = R.params_to_device(g)
    m = torch.tensor(med.as_array(), device="cuda")
    st = renderer.state()
    img, depth, _ = renderer.forward(st, p, m, cam)
    fT = renderer.state_array(st, "final_T", torch.float32, (cam.height, cam.width))
    restored = renderer.restore(img, depth, m)
    clean = renderer.render_clean(p, cam)[0]
    opaque = (fT < 1e-3).cpu().numpy()
    diff = (restored - clean).cpu().numpy()[:, opaque]
    psnr = -10 * np.log10(np.mean(diff ** 2))
    print({"opaque_fraction": float(opaque.mean()), "psnr_db": float(psnr)})
    assert opaque.mean() > 0.3 and psnr > 30.0
