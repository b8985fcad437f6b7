"""The fused training-step backward (gradients + Adam in place) against the
oracle's FP64 gradients followed by the oracle's textbook Adam step, and
against the unfused GPU path (backward, then splash_adam_step)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adam as oadam
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import compare_forward, gpu_forward, upstream_keep
from test_gpu_forward import _box_scene

pytestmark = pytest.mark.gpu

LR = {"means": 1.6e-4, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "sh": 2.5e-3, "medium": 2.5e-3}
NAMES = R.PARAM_NAMES + ("medium",)


def _moments(rng, shapes):
    m = {k: rng.normal(0, 1e-3, s).astype(np.float32) for k, s in shapes.items()}
    v = {k: rng.uniform(1e-5, 1e-3, s).astype(np.float32) for k, s in shapes.items()}
    return m, v


@pytest.mark.parametrize("scene", ["tiny", "box3"])
def test_fused_step_matches_oracle_gradient_then_adam(cuda_lib, scene):
    if scene == "tiny":
        g, med, cam = scenes.tiny_scene(0)
    else:
        g, med, cam = _box_scene(91, 1500, 90, 70, 80.0, 3, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    r = R.Renderer()
    out = gpu_forward(r, g, med, cam)
    ora = oracle.render(g, med, cam)
    fwd = compare_forward(out, ora, label=f"fused step {scene}", scene=(g, med, cam))
    rng = np.random.default_rng(5)
    keep = upstream_keep(ora, fwd)
    G = (rng.standard_normal((3, cam.height, cam.width)) * keep).astype(np.float32)
    shapes = {k: getattr(g, k).shape for k in R.PARAM_NAMES}
    shapes["medium"] = (9,)
    m0, v0 = _moments(rng, shapes)
    step = 5
    md = {k: torch.from_numpy(m0[k].copy()).cuda() for k in NAMES}
    vd = {k: torch.from_numpy(v0[k].copy()).cuda() for k in NAMES}
    gmed = torch.empty(9, device="cuda")
    r.backward_adam(out["state"], out["params"], out["medium"], cam, torch.from_numpy(G).cuda(), md, vd, LR, step,
                    medium_min=None, grad_medium=gmed)
    torch.cuda.synchronize()
    ref = oracle.backward(g, med, cam, G.astype(np.float64), branch=fwd["branch"])
    p0 = {k: getattr(g, k).astype(np.float64) for k in R.PARAM_NAMES}
    p0["medium"] = med.as_array().astype(np.float64)
    for k in NAMES:
        exp_p, exp_m, exp_v = oadam.adam_step(p0[k], ref[k], m0[k], v0[k], step, LR[k])
        got_p = (out["params"][k] if k != "medium" else out["medium"]).cpu().numpy()
        # the parameter moves by lr * (m-hat / sqrt(v-hat)): compare the moves
        dp_exp, dp_got = exp_p - p0[k], got_p.astype(np.float64) - p0[k]
        tol = 2e-3 * np.abs(dp_exp) + 2e-3 * LR[k] * 1e-2 + 1e-6 * np.abs(p0[k])
        bad = np.abs(dp_got - dp_exp) > tol
        assert not bad.any(), (k, int(bad.sum()), dp_got.reshape(-1)[:4], dp_exp.reshape(-1)[:4])
        np.testing.assert_allclose(md[k].cpu().numpy(), exp_m, rtol=2e-3, atol=1e-3 * np.abs(exp_m).max() + 1e-12)
    np.testing.assert_allclose(gmed.cpu().numpy(), ref["medium"], rtol=1e-3, atol=1e-5 * np.abs(ref["medium"]).max())


def test_fused_step_matches_unfused_gpu_path(cuda_lib):
    """Same step two ways on the 300k scene: fused kernel vs backward + multi-group Adam."""
    g, med, cam = scenes.mid_scene()
    r = R.Renderer()
    rng = np.random.default_rng(7)
    G = torch.tensor(rng.standard_normal((3, cam.height, cam.width)) * 1e-3, dtype=torch.float32, device="cuda")
    results = []
    for fused in (True, False):
        out = gpu_forward(r, g, med, cam)
        p = dict(out["params"])
        tens = {k: p[k] for k in R.PARAM_NAMES}
        tens["medium"] = out["medium"]
        # non-zero moments keep the update a smooth function of the gradient
        # (atomics order makes the two gradients differ in the last bits)
        mrng = np.random.default_rng(11)
        md = {k: torch.from_numpy(mrng.normal(0, 1e-4, tuple(t.shape)).astype(np.float32)).cuda() for k, t in tens.items()}
        vd = {k: torch.from_numpy(mrng.uniform(1e-6, 1e-5, tuple(t.shape)).astype(np.float32)).cuda()
              for k, t in tens.items()}
        if fused:
            r.backward_adam(out["state"], p, out["medium"], cam, G, md, vd, LR, 3)
        else:
            grads = r.backward(out["state"], p, out["medium"], cam, G)
            R.adam_step([{"param": tens[k], "grad": grads[k], "m": md[k], "v": vd[k], "lr": LR[k],
                          "clamp_min": 0.0 if k == "medium" else None} for k in NAMES], 3)
        torch.cuda.synchronize()
        results.append({k: tens[k].cpu().numpy() for k in NAMES} | {"m_" + k: md[k].cpu().numpy() for k in NAMES})
    a, b = results
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-4, atol=1e-5 * np.abs(b[k]).max() + 1e-9)


def test_fused_step_at_full_size_matches_oracle_gradient_then_adam(cuda_lib):
    """The fused adjoint + Adam at the bench's size (1.5M Gaussians, SH 3,
    1920x1280): the upstream gradient is non-zero at 200 sampled pixels only,
    so the oracle's exact gradient needs just those pixels; every parameter,
    moment and the nine medium gradients of the step are then compared with
    the oracle gradient followed by the textbook Adam step."""
    g, med, cam = scenes.full_scene()
    r = R.Renderer()
    out = gpu_forward(r, g, med, cam)
    rng = np.random.default_rng(13)
    pix = rng.choice(cam.width * cam.height, 200, replace=False)
    ora = oracle.render(g, med, cam, pix=pix)
    fwd = compare_forward(out, ora, pix=pix, label="fused step full", scene=(g, med, cam))
    keep = upstream_keep(ora, fwd)
    H, W = cam.height, cam.width
    Gs = np.float64(np.float32(rng.standard_normal((3, pix.size)) * keep))
    G = np.zeros((3, H * W), np.float32)
    G[:, pix] = Gs
    shapes = {k: getattr(g, k).shape for k in R.PARAM_NAMES}
    shapes["medium"] = (9,)
    m0, v0 = _moments(rng, shapes)
    step = 7
    md = {k: torch.from_numpy(m0[k].copy()).cuda() for k in NAMES}
    vd = {k: torch.from_numpy(v0[k].copy()).cuda() for k in NAMES}
    gmed = torch.empty(9, device="cuda")
    r.backward_adam(out["state"], out["params"], out["medium"], cam, torch.from_numpy(G.reshape(3, H, W)).cuda(),
                    md, vd, LR, step, medium_min=None, grad_medium=gmed)
    torch.cuda.synchronize()
    ref = oracle.backward(g, med, cam, Gs, pix=pix, branch=fwd["branch"])
    assert np.abs(ref["means"]).sum() > 0
    p0 = {k: getattr(g, k).astype(np.float64) for k in R.PARAM_NAMES}
    p0["medium"] = med.as_array().astype(np.float64)
    for k in NAMES:
        exp_p, exp_m, exp_v = oadam.adam_step(p0[k], ref[k], m0[k], v0[k], step, LR[k])
        got_p = (out["params"][k] if k != "medium" else out["medium"]).cpu().numpy()
        dp_exp, dp_got = exp_p - p0[k], got_p.astype(np.float64) - p0[k]
        tol = 2e-3 * np.abs(dp_exp) + 2e-3 * LR[k] * 1e-2 + 1e-6 * np.abs(p0[k])
        bad = np.abs(dp_got - dp_exp) > tol
        assert not bad.any(), (k, int(bad.sum()), dp_got.reshape(-1)[bad.reshape(-1)][:4], dp_exp.reshape(-1)[bad.reshape(-1)][:4])
        np.testing.assert_allclose(md[k].cpu().numpy(), exp_m, rtol=2e-3, atol=1e-3 * np.abs(exp_m).max() + 1e-12)
    np.testing.assert_allclose(gmed.cpu().numpy(), ref["medium"], rtol=1e-3, atol=1e-5 * np.abs(ref["medium"]).max())
