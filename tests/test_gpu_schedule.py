"""The appendix's training schedule on the GPU: the opacity reset kernel
against the oracle, and the fit loop applying the position learning rate
and the resets on schedule."""
import numpy as np
import pytest
import torch

from oracle import schedule as OS
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes, schedule, warmstart

pytestmark = pytest.mark.gpu


def test_opacity_reset_matches_oracle(cuda_lib):
    rng = np.random.default_rng(0)
    cap = OS.opacity_reset(np.array([1e9]))[0][0]  # the oracle's FP64 cap
    for n in (1, 1000, 300_001):
        lg = rng.normal(0, 3, n).astype(np.float32)
        lg[: min(n, 3)] = np.array([-4.6, -4.59, cap], np.float32)[: min(n, 3)]
        m = torch.ones(n, device="cuda")
        v = torch.ones(n, device="cuda")
        t = torch.from_numpy(lg).cuda()
        R.opacity_reset(t, m, v, 0.01)
        got = t.cpu().numpy()
        want = OS.opacity_reset(lg)[0]
        below = lg.astype(np.float64) < cap - 1e-5
        assert np.array_equal(got[below], lg[below])               # untouched, bit for bit
        np.testing.assert_array_max_ulp(got, np.float32(want), maxulp=1)  # capped: the cap in FP32
        assert float(m.abs().max()) == 0.0 and float(v.abs().max()) == 0.0


def test_schedule_matches_oracle():
    for t in (0, 1, 999, 15_000, 29_999, 30_000, 50_000):
        assert schedule.position_lr(t) == pytest.approx(OS.position_lr(t), rel=1e-14)


def test_fit_applies_the_schedule(cuda_lib):
    r = R.Renderer()
    g, med, _ = scenes.patch_scene(30_000, 4, (2.0, 12.0), 320, 214, 300.0)
    cams = scenes.arc_cameras(8, 4, width=320, height=214, fx=300.0)
    gt = R.params_to_device(g)
    m = torch.tensor(med.as_array(), device="cuda")
    tgt = [r.render(gt, m, c)[0].clone() for c in cams]
    fit = warmstart.Fit(r, gt, warmstart.DEFAULT_MEDIUM, cams, tgt, schedule=True, reset_every=4)
    for _ in range(9):
        fit.step()
        assert fit.lr["means"] == schedule.position_lr(fit.it - 1)
    r.sync_status()
    assert fit.resets_done == 2  # at iterations 4 and 8
    p = torch.sigmoid(fit.params["opacity_logits"])
    # one Adam step since the last reset: every opacity is near or below 1 %
    assert float(p.max()) < 0.02
