"""The MCMC densification kernels (Sec. IV-D: the sampling form of
3DGS-MCMC the paper adopts) against their FP64 oracle, through the C ABI:
which Gaussians are dead, which source each draws, the shared opacity and
scale of a source and its copies, the zeroed moments, and the position
noise."""
import math

import numpy as np
import pytest
import torch

from oracle import mcmc as OM
from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import render as R

pytestmark = pytest.mark.gpu

MARGIN = 1e-6  # a dead / live decision this close (relative) to the threshold may go either way


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


def _set(n, rng, dead_frac, deg=3):
    k = (deg + 1) ** 2
    logits = rng.normal(0.5, 1.5, n)
    dead = rng.random(n) < dead_frac
    logits[dead] = rng.uniform(-12.0, math.log(0.005 / 0.995), dead.sum())
    p = {"means": rng.normal(0, 2, (n, 3)), "log_scales": rng.normal(-4.0, 0.8, (n, 3)),
         "quats": rng.normal(0, 1, (n, 4)), "opacity_logits": logits, "sh": rng.normal(0, 0.5, (n, k, 3))}
    p = {k2: v.astype(np.float32) for k2, v in p.items()}
    mo = {k2: rng.normal(0, 1e-3, v.shape).astype(np.float32) for k2, v in p.items()}
    ve = {k2: rng.uniform(0, 1e-5, v.shape).astype(np.float32) for k2, v in p.items()}
    u = rng.random(n).astype(np.float32)
    return p, mo, ve, u


def _gpu(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


@pytest.mark.parametrize("n,dead_frac", [(1, 0.0), (777, 0.3), (20_000, 0.1), (300_001, 0.05)])
def test_relocation_matches_oracle(renderer, n, dead_frac):
    rng = np.random.default_rng(n)
    p, mo, ve, u = _set(n, rng, dead_frac)
    assert (OM.dead_margins(p["opacity_logits"]) < MARGIN).sum() == 0  # no decision at FP64 resolution here
    gp, gm, gv = _gpu(p), _gpu(mo), _gpu(ve)
    gp["sh_degree"] = 3
    nd = R.mcmc_relocate(renderer, gp, gm, gv, torch.from_numpy(u).cuda())
    renderer.sync_status()
    P, M, V, n_dead = OM.relocate(p, mo, ve, u.astype(np.float64))
    assert nd == n_dead
    for k in R.PARAM_NAMES:
        got = gp[k].cpu().numpy()
        want = P[k]
        if k in ("opacity_logits", "log_scales"):
            # computed in FP64 on both sides, rounded once to FP32: equal to 1 ulp
            np.testing.assert_allclose(got, want, rtol=2.4e-7, atol=1e-30, err_msg=k)
        else:
            np.testing.assert_array_equal(got, np.float32(want), err_msg=k)
        np.testing.assert_array_equal(gm[k].cpu().numpy(), np.float32(M[k]), err_msg="m " + k)
        np.testing.assert_array_equal(gv[k].cpu().numpy(), np.float32(V[k]), err_msg="v " + k)


def test_relocation_of_popular_sources_caps_at_51(renderer):
    """Two live Gaussians and 300 dead ones: each source is drawn about 150
    times and stands for N = 51 Gaussians (the cap); every dead one ends as
    a copy of one of the two sources."""
    rng = np.random.default_rng(5)
    p, mo, ve, u = _set(302, rng, 0.0)
    p["opacity_logits"][2:] = np.float32(-9.0)
    p["opacity_logits"][:2] = np.float32([1.5, 0.5])
    gp, gm, gv = _gpu(p), _gpu(mo), _gpu(ve)
    gp["sh_degree"] = 3
    assert R.mcmc_relocate(renderer, gp, gm, gv, torch.from_numpy(u).cuda()) == 300
    P, _, _, _ = OM.relocate(p, mo, ve, u.astype(np.float64))
    got = gp["opacity_logits"].cpu().numpy()
    np.testing.assert_allclose(got, P["opacity_logits"], rtol=2.4e-7)
    o_new, _ = OM.shared_opacity_scale(1 / (1 + math.exp(-1.5)), 51)
    assert 1 / (1 + math.exp(-float(got[0]))) == pytest.approx(o_new, rel=1e-6)
    means = gp["means"].cpu().numpy()
    assert all((means[i] == means[0]).all() or (means[i] == means[1]).all() for i in range(2, 302))


def test_relocation_without_dead_or_live(renderer):
    rng = np.random.default_rng(6)
    for logit in (3.0, -9.0):  # nothing dead; everything dead (nothing to draw from)
        p, mo, ve, u = _set(1000, rng, 0.0)
        p["opacity_logits"][:] = np.float32(logit)
        gp, gm, gv = _gpu(p), _gpu(mo), _gpu(ve)
        gp["sh_degree"] = 3
        nd = R.mcmc_relocate(renderer, gp, gm, gv, torch.from_numpy(u).cuda())
        assert nd == (0 if logit > 0 else 1000)
        for k in R.PARAM_NAMES:
            np.testing.assert_array_equal(gp[k].cpu().numpy(), p[k])
            np.testing.assert_array_equal(gm[k].cpu().numpy(), mo[k])


def test_noise_matches_oracle(renderer):
    rng = np.random.default_rng(7)
    n = 50_000
    p, _, _, _ = _set(n, rng, 0.2)
    p["log_scales"] = np.float32(rng.normal(-2.0, 0.5, (n, 3)))
    eta = rng.standard_normal((n, 3)).astype(np.float32)
    gp = _gpu(p)
    R.mcmc_noise(gp, torch.from_numpy(eta).cuda(), lr=1.6e-4, lambda_noise=5e5)
    torch.cuda.synchronize()
    want = OM.noise(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], eta, 1.6e-4, 5e5)
    got = gp["means"].cpu().numpy().astype(np.float64)
    step = want - p["means"].astype(np.float64)
    # FP32 arithmetic of the step (exp, rotation, products) against FP64, plus the FP32 sum
    tol = 1e-5 * np.abs(step).max(axis=1, keepdims=True) + 2 * 6e-8 * np.abs(want)
    assert (np.abs(got - want) <= tol).all()
    assert np.abs(step).max() > 1e-4  # the transparent ones move


def test_argument_checks(renderer):
    L = _abi.lib()
    nd = __import__("ctypes").c_int64()
    assert L.splash_mcmc_relocate(renderer._ctx, None, None, None, 10, 3, None, 0.005, None, None) == _abi.ERR_INVALID_ARG
    assert L.splash_mcmc_noise(None, None, None, None, None, -1, 1.0, 1.0, None) == _abi.ERR_INVALID_ARG
    del nd


def test_fit_relocates_on_schedule(cuda_lib):
    """The fit with MCMC densification: noise after every step, relocation at
    every 3rd iteration in [3, 10); a fifth of the Gaussians start dead, so
    the first relocation moves them and the count stays fixed."""
    from paper_2411_19588_b300 import scenes, warmstart
    r = R.Renderer()
    g, med, _ = scenes.patch_scene(20_000, 6, (2.0, 12.0), 320, 214, 300.0)
    cams = scenes.arc_cameras(8, 6, width=320, height=214, fx=300.0)
    gt = R.params_to_device(g)
    m = torch.tensor(med.as_array(), device="cuda")
    tgt = [r.render(gt, m, c)[0].clone() for c in cams]
    start, _ = scenes.perturb(g, med, seed=7)
    p = R.params_to_device(start)
    p["opacity_logits"][::5] = -9.0
    fit = warmstart.Fit(r, p, warmstart.DEFAULT_MEDIUM, cams, tgt,
                        mcmc={"start": 3, "stop": 10, "every": 3})
    losses = [fit.step().item() for _ in range(12)]
    r.sync_status()
    assert fit.relocations == 3  # at iterations 3, 6 and 9
    assert fit.dead_relocated[0] >= 4000
    assert fit.params["means"].shape[0] == 20_000
    assert all(math.isfinite(x) for x in losses)
    assert float(torch.sigmoid(fit.params["opacity_logits"]).min()) > 0.0
