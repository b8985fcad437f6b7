"""The training-step kernels against their oracles: L1 + 0.2 (1 - SSIM) with
its gradient, and the multi-group Adam step."""
import numpy as np
import pytest
import torch

from oracle import adam as oadam
from oracle import loss as oloss
from paper_2411_19588_b300 import render as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


# 100x128: rows a multiple of 4 floats, so tiles whose haloed window lies inside the image
# take the 16-byte load path and the others the checked one; "mis" offsets both buffers by
# 4 bytes, which sends every tile down the checked path
@pytest.mark.parametrize("C,H,W,mis", [(3, 130, 170, 0), (3, 16, 32, 0), (1, 45, 7, 0), (3, 100, 128, 0),
                                       (3, 100, 128, 1), (3, 1280, 1920, 0)])
def test_loss_and_gradient_match_oracle(renderer, C, H, W, mis):
    rng = np.random.default_rng(C * H + W)
    x = rng.uniform(0, 1, (C, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1).astype(np.float32)
    st = renderer.state()

    def dev(a):
        if not mis:
            return torch.from_numpy(a).cuda()
        buf = torch.empty(a.size + 1, device="cuda")
        buf[1:] = torch.from_numpy(a.ravel()).cuda()
        return buf[1:].view(a.shape)

    loss, grad = renderer.loss(st, dev(x), dev(y), 0.2)
    torch.cuda.synchronize()
    if H * W > 1_000_000:  # the oracle on a crop far from the borders is exact for interior pixels
        ref_l, ref_g = oloss.loss_and_grad(x[:, 600:700, 900:1000], y[:, 600:700, 900:1000], 0.2)
        assert np.isfinite(loss.item())
        # interior pixels of the crop see the same windows in both
        g = grad.cpu().numpy()[:, 610:690, 910:990] * (H * W) / (100 * 100)
        np.testing.assert_allclose(g, ref_g[:, 10:90, 10:90], rtol=2e-3, atol=2e-3 * np.abs(ref_g).max())
        return
    ref_l, ref_g = oloss.loss_and_grad(x, y, 0.2)
    assert abs(loss.item() - ref_l) < 2e-6 * max(1.0, abs(ref_l))
    g = grad.cpu().numpy()
    np.testing.assert_allclose(g, ref_g, rtol=1e-3, atol=1e-4 * np.abs(ref_g).max())


def test_adam_matches_oracle(cuda_lib):
    rng = np.random.default_rng(9)
    sizes = [4_500_003, 1000, 7, 4096 * 3]
    lrs = [1.6e-4, 5e-3, 2.5e-3, 0.05]
    ps = [rng.standard_normal(n).astype(np.float32) for n in sizes]
    ms = [np.zeros(n, np.float32) for n in sizes]
    vs = [np.zeros(n, np.float32) for n in sizes]
    dp = [torch.from_numpy(p).cuda() for p in ps]
    dm = [torch.from_numpy(m).cuda() for m in ms]
    dv = [torch.from_numpy(v).cuda() for v in vs]
    refs = [(p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)) for p, m, v in zip(ps, ms, vs)]
    for step in range(1, 4):
        gs = [rng.standard_normal(n).astype(np.float32) for n in sizes]
        dg = [torch.from_numpy(g).cuda() for g in gs]
        groups = [{"param": dp[i], "grad": dg[i], "m": dm[i], "v": dv[i], "lr": lrs[i],
                   "clamp_min": 0.0 if i == 2 else None} for i in range(len(sizes))]
        R.adam_step(groups, step)
        refs = [oadam.adam_step(refs[i][0], gs[i], refs[i][1], refs[i][2], step, lrs[i],
                                clamp_min=0.0 if i == 2 else None) for i in range(len(sizes))]
    torch.cuda.synchronize()
    for i in range(len(sizes)):
        np.testing.assert_allclose(dp[i].cpu().numpy(), refs[i][0], rtol=1e-5, atol=1e-6 * lrs[i] * 10)
        np.testing.assert_allclose(dm[i].cpu().numpy(), refs[i][1], rtol=1e-5, atol=1e-7)
