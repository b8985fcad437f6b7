"""GPU parity of the densification step (appendix schedule; the 3DGS
procedure): the statistics gathered by the fused training step, the plan
(prune / keep / clone / split) and the new arrays, against the FP64 oracle;
and the fit loop densifying on its schedule."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import densify as OD
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes, warmstart

from parity import compare_forward, gpu_forward, medium_tensor, upstream_keep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


def test_statistics_match_the_oracle_screen_gradients(renderer):
    g, m, cam = scenes.tiny_scene(3)
    out = gpu_forward(renderer, g, m, cam)
    st, params, med = out["state"], out["params"], out["medium"]
    ora = oracle.render(g, m, cam)
    fwd = compare_forward(out, ora, label="densify stats", scene=(g, m, cam))
    keep = upstream_keep(ora, fwd)
    G = np.float64(np.float32(np.random.default_rng(3).standard_normal((3, cam.height, cam.width)) * keep))
    names = R.PARAM_NAMES + ("medium",)
    tens = dict(params)
    tens["medium"] = med
    mo = {k: torch.zeros_like(tens[k]) for k in names}
    ve = {k: torch.zeros_like(tens[k]) for k in names}
    stats = torch.zeros((g.n, 2), device="cuda")
    stats[:, 0] = 0.5  # accumulates (+=)
    renderer.backward_adam(st, params, med, cam, torch.tensor(G, dtype=torch.float32, device="cuda"), mo, ve,
                           warmstart.FIT_LR, 1, densify_stats=stats)
    got = stats.cpu().numpy().astype(np.float64)
    ref = oracle.backward(g, m, cam, G, branch=fwd["branch"])
    # in the view: inside (z_near, z_far] and opaque enough ever to reach alpha >= 1/255
    vis = (oracle.project(g, m, cam)["vis"] > 0) & (1 / (1 + np.exp(-g.opacity_logits.astype(np.float64))) >= 1 / 255)
    want = OD.stat_increment(ref["proj"][:, 0:2], cam.width, cam.height)
    assert np.array_equal(got[:, 1], vis.astype(np.float64))           # in-view count
    np.testing.assert_allclose(got[vis, 0] - 0.5, want[vis], rtol=1e-3, atol=1e-5 * want.max())
    assert np.all(got[~vis, 0] == 0.5)


def _random_set(n, rng, deg=3):
    k = (deg + 1) ** 2
    p = {"means": rng.normal(0, 2, (n, 3)), "log_scales": rng.normal(-4.0, 0.8, (n, 3)),
         "quats": rng.normal(0, 1, (n, 4)), "opacity_logits": rng.normal(-1.0, 2.0, n),
         "sh": rng.normal(0, 0.5, (n, k, 3))}
    p = {k2: v.astype(np.float32) for k2, v in p.items()}
    mo = {k2: rng.normal(0, 1e-3, v.shape).astype(np.float32) for k2, v in p.items()}
    ve = {k2: rng.uniform(0, 1e-5, v.shape).astype(np.float32) for k2, v in p.items()}
    stats = np.stack([rng.uniform(0, 0.01, n), rng.integers(0, 30, n)], 1).astype(np.float32)
    return p, mo, ve, stats


DMARGIN = 1e-5   # a decision this close (relative) to its threshold may go either way in FP32


def _edge_set(rng):
    """64 Gaussians, a quarter of them on a threshold at FP32 resolution:
    logit = fl32(logit(0.1)), max log-scale = fl32(log(dense)), mean
    gradient fl32(threshold); the FP64 definitions decide these by the
    rounding of the stored values."""
    p, mo, ve, stats = _random_set(64, rng)
    dense = 0.01 * 3.0
    for i in range(0, 64, 4):
        j = i // 4 % 3
        if j == 0:
            p["opacity_logits"][i] = np.float32(math.log(0.1 / 0.9))
        elif j == 1:
            p["log_scales"][i] = np.float32(math.log(dense)) - np.float32([0.5, 0.0, 0.7])
            stats[i] = [0.01, 10]
            p["opacity_logits"][i] = 2.0
        else:
            stats[i] = [np.float32(0.0002) * 7, 7]
            p["opacity_logits"][i] = 2.0
    return p, mo, ve, stats


@pytest.mark.parametrize("n", [1, 777, 20_000, "edge"])
def test_plan_and_apply_match_oracle(renderer, n):
    """The oracle decides in FP64 on the definitions; a decision within
    DMARGIN of its threshold is accepted either way (its Gaussians counted).
    Every other decision, and every output value, must match exactly."""
    rng = np.random.default_rng(5 if n == "edge" else n)
    p, mo, ve, stats = _edge_set(rng) if n == "edge" else _random_set(n, rng)
    n = len(p["opacity_logits"])
    noise = rng.standard_normal((n, 2, 3)).astype(np.float32)
    extent = 3.0
    t = lambda d: {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}
    gp, gm, gv = t(p), t(mo), t(ve)
    gp["sh_degree"] = 3
    P, M, V = R.densify(renderer, gp, gm, gv, torch.from_numpy(stats).cuda(), torch.from_numpy(noise).cuda(), extent)
    renderer.sync_status()
    got = {k: P[k].cpu().numpy() for k in R.PARAM_NAMES}
    cls = dict(dense=0.01 * extent)
    margins = OD.decision_margins(p["log_scales"], p["opacity_logits"], stats, **cls)
    near = margins < DMARGIN
    print(f"densify n={n}: {int(near.any(1).sum())} Gaussians with a near decision")
    act0 = OD.classify(p["log_scales"], p["opacity_logits"], stats, **cls)
    if n > 100:
        assert set(np.unique(act0)) == {OD.PRUNE, OD.KEEP, OD.CLONE, OD.SPLIT}
    gm_, gv_ = ({k: M[k].cpu().numpy() for k in R.PARAM_NAMES}, {k: V[k].cpu().numpy() for k in R.PARAM_NAMES})
    # Outputs are consecutive per input Gaussian, so each Gaussian is checked
    # at the cursor: its FP64 action, or, for a near decision, any outcome of
    # its near decisions, must reproduce the GPU's rows exactly (split
    # samples, computed in FP32, within 2e-6).
    cursor = 0
    for i in range(n):
        bits = [1 << j for j in range(3) if near[i, j]]
        cands = []
        for combo in range(1 << len(bits)):
            f = sum(b for t, b in enumerate(bits) if (combo >> t) & 1)
            flip = np.zeros(n, np.int64)
            flip[i] = f
            cands.append(OD.classify(p["log_scales"][i:i + 1], p["opacity_logits"][i:i + 1], stats[i:i + 1],
                                     flip=flip[i:i + 1], **cls)[0])
        if not bits:
            assert cands == [act0[i]]
        ok = False
        # longest output first: a keep's row is also a clone's first row, and a
        # prune (no rows) always "matches"
        for a in sorted(dict.fromkeys(cands), key=lambda a: {OD.PRUNE: 2, OD.KEEP: 1}.get(int(a), 0)):
            one = {k: p[k][i:i + 1] for k in R.PARAM_NAMES}
            oP, oM, oV = OD.apply(one, {k: mo[k][i:i + 1] for k in R.PARAM_NAMES},
                                  {k: ve[k][i:i + 1] for k in R.PARAM_NAMES}, np.array([a]), noise[i:i + 1])
            rows = oP["means"].shape[0]
            if cursor + rows > got["means"].shape[0]:
                continue
            sl = slice(cursor, cursor + rows)
            good = True
            for k in R.PARAM_NAMES:
                if a == OD.SPLIT and k in ("means", "log_scales"):
                    good &= np.allclose(got[k][sl], oP[k], rtol=2e-6, atol=2e-6)
                else:
                    good &= np.array_equal(got[k][sl], np.float32(oP[k]))
                good &= np.array_equal(gm_[k][sl], np.float32(oM[k])) and np.array_equal(gv_[k][sl], np.float32(oV[k]))
            if good:
                ok = True
                cursor += rows
                break
        assert ok, (i, cands, near[i], margins[i])
    assert cursor == got["means"].shape[0]


def test_fit_densifies_on_schedule(renderer):
    g, med, _ = scenes.patch_scene(20_000, 6, (2.0, 12.0), 320, 214, 300.0)
    cams = scenes.arc_cameras(8, 6, width=320, height=214, fx=300.0)
    gt = R.params_to_device(g)
    m = torch.tensor(med.as_array(), device="cuda")
    tgt = [renderer.render(gt, m, c)[0].clone() for c in cams]
    start, _ = scenes.perturb(g, med, seed=7)
    fit = warmstart.Fit(renderer, R.params_to_device(start), warmstart.DEFAULT_MEDIUM, cams, tgt,
                        densify={"start": 2, "stop": 9, "every": 3, "grad_threshold": 1e-4})
    losses = [fit.step().item() for _ in range(12)]
    renderer.sync_status()
    assert fit.densify_steps == 2 and len(fit.counts) == 3   # at iterations 3 and 6 (9 is past stop)
    assert fit.counts[1] != fit.counts[0]
    assert all(math.isfinite(x) for x in losses)
    assert fit.params["means"].shape[0] == fit.m["means"].shape[0] == fit.counts[-1]
