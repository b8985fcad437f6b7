"""GPU parity of the backscatter estimate and the L_best prior (Sec. IV-B,
Eq. 7-9; Alg. 1 and Alg. 2) against the FP64 oracle, through the C ABI.

Integer work (resized FP32 maps, cluster membership, kept pixels, fit
points) must match bit for bit: both sides round the same exact area means
once to FP32 and take every decision on those values. The fit is compared
on its residual and, where the minimum is unique, on the parameters."""
import numpy as np
import pytest
import torch

from oracle import backscatter as BS
from paper_2411_19588_b300 import backscatter as GB
from paper_2411_19588_b300 import render as R
from tests import water

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    r = R.Renderer()
    yield r
    r.close()


def _run(renderer, img, depth, **opts):
    H, W = depth.shape
    o = dict(GB.DEFAULTS)
    o.update(opts)
    w, h = GB.resized_size(W, H, o["resized_height"])
    resized = torch.empty((4, h, w), device="cuda")
    dark = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    res = GB.estimate(renderer, torch.from_numpy(np.ascontiguousarray(img)).cuda(),
                      torch.from_numpy(np.ascontiguousarray(depth)).cuda(), resized=resized, dark=dark, **opts)
    renderer.sync_status()
    return GB.read(res), resized.cpu().numpy(), dark.cpu().numpy().ravel().astype(bool)


def _oracle(img, depth, **opts):
    o = dict(GB.DEFAULTS)
    o.update(opts)
    img_s = BS.resize(img, o["resized_height"])
    z_s = BS.resize(np.asarray(depth)[None], o["resized_height"])[0]
    keep, _, _ = BS.dark_mask(img_s, z_s, o["p_dark"], o["edges"])
    pts = BS.depth_minima(img_s, z_s, keep, o["intervals"])
    fits = [BS.fit_channel(z, m, o["b_max"], o["beta_max"]) for z, m in pts]
    return img_s, z_s, keep, pts, fits


def _check(gpu, resized, dark, ora, unique=True, label=""):
    img_s, z_s, keep, pts, fits = ora
    assert np.array_equal(resized[:3], img_s), f"{label}: resized image differs"
    assert np.array_equal(resized[3], z_s), f"{label}: resized depth differs"
    assert np.array_equal(dark, keep), f"{label}: kept pixels differ ({dark.sum()} vs {keep.sum()})"
    assert gpu["n_dark"] == keep.sum()
    for k in range(3):
        gz, gv = gpu["points"][k]
        oz, ov = pts[k]
        assert np.array_equal(gz.astype(np.float64), oz) and np.array_equal(gv.astype(np.float64), ov), \
            f"{label}: points of channel {k} differ"
        B, beta, S = fits[k]
        gB, gbeta, gS = float(gpu["b_inf"][k]), float(gpu["beta_b"][k]), float(gpu["residual"][k])
        assert 0.0 <= gB <= 1.0 and 0.0 <= gbeta <= 5.0
        # the GPU minimum is no worse than the oracle's (float32 parameters)
        assert BS.residual(gB, gbeta, oz, ov) <= S * (1 + 1e-5) + 1e-11, f"{label}: channel {k} residual"
        assert gS == pytest.approx(S, rel=1e-4, abs=1e-11)
        if unique and _well_determined(oz, ov, beta, S):
            assert gbeta == pytest.approx(beta, rel=2e-5, abs=1e-6), f"{label}: beta of channel {k}"
            assert gB == pytest.approx(B, rel=2e-5, abs=1e-6), f"{label}: B_inf of channel {k}"


def _profile(z, m, beta):
    """Residual with the best B in [0, 1] for this beta (FP64)."""
    f = 1.0 - np.exp(-beta * z)
    ff = f @ f
    B = min(1.0, max(0.0, (m @ f) / ff)) if ff > 0 else 0.0
    return BS.residual(B, beta, z, m)


def _well_determined(z, m, beta, S):
    """The parameters are compared only where the residual pins them: moving
    beta by 0.1% (inside the box) must raise the profiled residual by more
    than FP32 can resolve (1e-5 relative); otherwise both answers are minima
    to FP32 resolution and the residual comparison above is the check."""
    rises = [_profile(z, m, b) - S for b in (beta * 0.999, beta * 1.001) if 0.0 <= b <= 5.0]
    return len(rises) == 2 and min(rises) > 1e-5 * S + 1e-12


@pytest.mark.parametrize("W,H,seed", [(1920, 1280, 11), (1280, 854, 12)])
def test_estimate_full_size_matches_oracle(renderer, W, H, seed):
    img, depth, _ = water.view(seed, W, H)
    gpu, resized, dark = _run(renderer, img, depth)
    assert (gpu["width"], gpu["height"]) == (450, 300)
    _check(gpu, resized, dark, _oracle(img, depth), label=f"{W}x{H}")


def test_estimate_recovers_the_medium(renderer):
    img, depth, med = water.view(5, 450, 300, shadow_block=4, shadow_frac=0.04)
    gpu, _, _ = _run(renderer, img, depth)
    np.testing.assert_allclose(gpu["b_inf"], med.b_inf, rtol=5e-5)
    np.testing.assert_allclose(gpu["beta_b"], med.beta_b, rtol=5e-5)


@pytest.mark.parametrize("W,H,opts", [
    (128, 96, {}),                                          # upsampled to 300 x 400
    (37, 23, {"resized_height": 16}),                       # ragged, one block
    (641, 427, {"edges": 3, "intervals": 2}),               # one interval: one point per channel
    (300, 200, {"p_dark": 1.0, "resized_height": 100}),     # every pixel kept
    (500, 333, {"edges": 65, "intervals": 65}),             # largest tables
    (9, 7, {"resized_height": 1}),                          # a single row
])
def test_estimate_edge_cases_match_oracle(renderer, W, H, opts):
    img, depth, _ = water.view(3, W, H)
    gpu, resized, dark = _run(renderer, img, depth, **opts)
    unique = opts.get("intervals", 25) > 2 and H > 20 and opts.get("resized_height", 300) > 1
    _check(gpu, resized, dark, _oracle(img, depth, **opts), unique=unique, label=str(opts))


def test_ties_and_constant_depth_match_oracle(renderer):
    """Constant colour: every darkness key ties, so the kept pixels are the
    first ceil(p n) of each cluster in index order; constant depth puts
    every pixel in the top cluster."""
    rng = np.random.default_rng(0)
    img = np.full((3, 600, 900), 0.25, np.float32)
    depth = rng.uniform(1, 9, (600, 900)).astype(np.float32)
    gpu, resized, dark = _run(renderer, img, depth)
    _check(gpu, resized, dark, _oracle(img, depth), unique=False, label="constant colour")
    depth = np.full((600, 900), 3.0, np.float32)
    img = rng.uniform(0, 1, (3, 600, 900)).astype(np.float32)
    gpu, resized, dark = _run(renderer, img, depth)
    _check(gpu, resized, dark, _oracle(img, depth), unique=False, label="constant depth")
    assert gpu["n_dark"] == int(np.ceil(0.01 * 300 * 450))


def test_options_are_validated(renderer):
    img = torch.zeros((3, 20, 30), device="cuda")
    depth = torch.ones((20, 30), device="cuda")
    from paper_2411_19588_b300 import _abi
    for bad in ({"edges": 1}, {"edges": 66}, {"intervals": 66}, {"p_dark": 0.0}, {"p_dark": 1.5},
                {"resized_height": 0}, {"beta_max": -1.0}):
        with pytest.raises(_abi.SplashError) as e:
            GB.estimate(renderer, img, depth, **bad)
        assert e.value.status == _abi.ERR_INVALID_ARG


def test_prior_loss_and_gradient(renderer):
    rng = np.random.default_rng(8)
    med = rng.uniform(0.05, 0.6, 9).astype(np.float32)
    pv = np.concatenate([rng.uniform(0.05, 0.6, 3), rng.uniform(0.05, 0.4, 3)]).astype(np.float32)
    pv[1] = med[4]                                  # one exact tie: sign 0
    g = torch.full((9,), 0.5, device="cuda")
    loss = torch.full((1,), 2.0, device="cuda")
    GB.prior(torch.from_numpy(med).cuda(), torch.from_numpy(pv).cuda(), 0.1, g, loss)
    want_l, want_g = BS.prior_loss_and_grad(med, pv[:3], pv[3:], 0.1)
    assert loss.item() == pytest.approx(2.0 + want_l, rel=1e-6)
    np.testing.assert_allclose(g.cpu().numpy(), 0.5 + want_g, rtol=0, atol=1e-7)
    assert want_g[4] == 0.0


def test_fused_adam_applies_the_prior(renderer):
    """backward_adam with a prior: the medium gradient it reports is the
    plain one plus lambda_est sign(medium - prior) on beta_B and B_inf."""
    from paper_2411_19588_b300 import scenes, warmstart
    g, _, cam = scenes.tiny_scene(1)
    params = R.params_to_device(g)
    medium0 = torch.tensor([0.2, 0.15, 0.1, 0.3, 0.25, 0.2, 0.15, 0.2, 0.3], device="cuda")
    pv = torch.tensor([0.5, 0.25, 0.1, 0.1, 0.3, 0.35], device="cuda")
    pv[1] = medium0[4]
    grads = []
    for prior in (None, pv):
        p = {k: (v.clone() if isinstance(v, torch.Tensor) else v) for k, v in params.items()}
        med = medium0.clone()
        names = R.PARAM_NAMES + ("medium",)
        tens = dict(p)
        tens["medium"] = med
        m = {k: torch.zeros_like(tens[k]) for k in names}
        v = {k: torch.zeros_like(tens[k]) for k in names}
        st = renderer.state()
        img, _, _ = renderer.forward(st, p, med, cam)
        dimg = torch.full_like(img, 1e-3)
        gm = torch.zeros(9, device="cuda")
        renderer.backward_adam(st, p, med, cam, dimg, m, v, warmstart.FIT_LR, 1, grad_medium=gm, prior=prior,
                               lambda_est=0.1)
        grads.append(gm.cpu().numpy())
    sign = np.sign(medium0.cpu().numpy()[3:] - pv.cpu().numpy())
    d = grads[1] - grads[0]
    # the two runs agree on beta_D up to the run-to-run rounding of the blend
    # backward's float atomics (a few ulp of the gradient), not bit for bit
    np.testing.assert_allclose(d[:3], 0.0, atol=1e-7 + 1e-6 * np.abs(grads[0][:3]).max())
    np.testing.assert_allclose(d[3:], 0.1 * sign, atol=1e-6 + 1e-6 * np.abs(grads[0][3:]).max())
    assert sign[1] == 0.0


def test_fit_re_estimates_on_schedule_and_tracks_the_water(renderer):
    """The fit with L_best re-estimates at iterations 0, 5, 10 (estimate_every
    = 5) from the iteration's target and the depth it just rendered; in
    between the prior stays fixed. (How close the estimate comes to the true
    water depends on the scene having unlit surfaces: the patch scenes have
    none, so only the bounds are checked here; the shadowed water views
    above check the recovery.)"""
    from paper_2411_19588_b300 import scenes, warmstart
    g, med, _ = scenes.patch_scene(60_000, 22, (2.0, 15.0), 480, 320, 450.0)
    cams = scenes.arc_cameras(20, 22, width=480, height=320, fx=450.0)
    gt = R.params_to_device(g)
    med_gt = torch.tensor(med.as_array(), device="cuda")
    tgt = [renderer.render(gt, med_gt, c)[0].clone() for c in cams]
    fit = warmstart.Fit(renderer, gt, warmstart.DEFAULT_MEDIUM, cams, tgt, lambda_est=0.1, estimate_every=5)
    priors = []
    for _ in range(12):
        fit.step()
        priors.append(GB.prior_of(fit.estimate).cpu().numpy().copy())
    renderer.sync_status()
    assert fit.estimates_done == 3
    for i in (1, 2, 3, 4, 6, 7, 8, 9, 11):
        assert np.array_equal(priors[i], priors[i - 1 if i not in (5, 10) else i])
    assert not np.array_equal(priors[4], priors[5]) and not np.array_equal(priors[9], priors[10])
    est = GB.read(fit.estimate)
    print({"beta_b": est["beta_b"].tolist(), "b_inf": est["b_inf"].tolist(), "true_beta_b": med.beta_b.tolist(),
           "true_b_inf": med.b_inf.tolist()})
    assert np.all((est["b_inf"] >= 0) & (est["b_inf"] <= 1)) and np.all((est["beta_b"] >= 0) & (est["beta_b"] <= 5))
    assert est["n_dark"] > 0 and min(est["n_points"]) > 0
