"""GPU parity of the pixel form of the water (Eq. 5 as printed, with the
Eq. 6 depth) against its FP64 oracle, forward and backward, through the C
ABI, with the comparison protocol of the segment form."""
import numpy as np
import pytest
import torch

from oracle import pixel as OP
from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import compare_forward, compare_grads, grads_to_numpy, medium_tensor, upstream_keep
from test_gpu_forward import _box_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


def _forward(renderer, g, m, cam):
    params = R.params_to_device(g)
    med = medium_tensor(m)
    st = renderer.state()
    img, depth, d01 = renderer.forward(st, params, med, cam, pixel=True)
    torch.cuda.synchronize()
    gpu = {"image": img.cpu().numpy().astype(np.float64), "depth": depth.cpu().numpy().astype(np.float64),
           "depth01": d01.cpu().numpy().astype(np.float64)}
    return gpu, st, params, med


@pytest.mark.parametrize("case", ["tiny", "ragged", "dense"])
def test_pixel_forward_matches_oracle(renderer, case):
    if case == "tiny":
        g, m, cam = scenes.tiny_scene(0)
    elif case == "ragged":
        g, m, cam = _box_scene(81, 1500, 100, 75, 90.0, 3, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    else:
        g, m, cam = _box_scene(82, 2500, 80, 60, 70.0, 3, log_scale=-1.7)
    gpu, _, _, _ = _forward(renderer, g, m, cam)
    ora = OP.render(g, m, cam)
    print(case, compare_forward(gpu, ora, label=f"pixel {case}", scene=(g, m, cam), branches=OP.branches))


def _upstream(rng, keep, H, W, depth=True):
    G = rng.standard_normal((3, H, W)) * keep
    Gz = rng.standard_normal((H, W)) * 0.05 * keep if depth else None
    G01 = rng.standard_normal((H, W)) * 0.3 * keep if depth else None
    f = lambda a: None if a is None else np.float64(np.float32(a))
    return f(G), f(Gz), f(G01)


@pytest.mark.parametrize("case,depth", [("tiny", True), ("ragged", True), ("dense", True), ("ragged", False)])
def test_pixel_backward_matches_oracle(renderer, case, depth):
    """Includes the dependence of z on every contributing Gaussian (through
    alpha and d) and the nine medium gradients."""
    if case == "tiny":
        g, m, cam = scenes.tiny_scene(0)
    elif case == "ragged":
        g, m, cam = _box_scene(83, 1500, 61, 47, 55.0, 1, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    else:
        g, m, cam = _box_scene(84, 2500, 80, 60, 70.0, 3, log_scale=-1.7)
    gpu, st, params, med = _forward(renderer, g, m, cam)
    ora = OP.render(g, m, cam)
    fwd = compare_forward(gpu, ora, label=f"pixel bwd {case} depth={depth}", scene=(g, m, cam), branches=OP.branches)
    G, Gz, G01 = _upstream(np.random.default_rng(5), upstream_keep(ora, fwd), cam.height, cam.width, depth)
    t = lambda a: None if a is None else torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    grads = renderer.backward(st, params, med, cam, t(G), t(Gz), t(G01), pixel=True)
    torch.cuda.synchronize()
    ref = OP.backward(g, m, cam, G, Gz, G01, branch=fwd["branch"])
    print(case, depth, compare_grads(grads_to_numpy(grads), ref, f"pixel {case}"))


def test_pixel_full_scene_sampled(renderer):
    """1.5M Gaussians at 1920x1280: sampled pixels forward, and an upstream
    gradient non-zero at 200 sampled pixels backward."""
    g, m, cam = scenes.full_scene()
    gpu, st, params, med = _forward(renderer, g, m, cam)
    rng = np.random.default_rng(9)
    pix = rng.choice(cam.width * cam.height, 200, replace=False)
    ora = OP.render(g, m, cam, pix=pix)
    fwd = compare_forward(gpu, ora, pix=pix, label="pixel full", scene=(g, m, cam), branches=OP.branches)
    keep = upstream_keep(ora, fwd)
    G = np.zeros((3, cam.height, cam.width))
    iy, ix = np.divmod(pix, cam.width)
    G[:, iy, ix] = np.float64(np.float32(rng.standard_normal((3, pix.size)) * keep))
    grads = renderer.backward(st, params, med, cam, torch.tensor(G, dtype=torch.float32, device="cuda"), pixel=True)
    torch.cuda.synchronize()
    ref = OP.backward(g, m, cam, G[:, iy, ix], pix=pix, branch=fwd["branch"])
    compare_grads(grads_to_numpy(grads), ref, "pixel full")


def test_pixel_state_checks(renderer):
    g, m, cam = scenes.tiny_scene(1)
    params = R.params_to_device(g)
    med = medium_tensor(m)
    G = torch.zeros((3, cam.height, cam.width), device="cuda")
    st = renderer.state()
    renderer.forward(st, params, med, cam)  # segment form
    with pytest.raises(_abi.SplashError) as e:
        renderer.backward(st, params, med, cam, G, pixel=True)
    assert e.value.status == _abi.ERR_STATE
    renderer.forward(st, params, med, cam, pixel=True)
    with pytest.raises(_abi.SplashError) as e:
        renderer.backward(st, params, med, cam, G)
    assert e.value.status == _abi.ERR_STATE
    renderer.backward(st, params, med, cam, G, pixel=True)
    renderer.sync_status()


def test_pixel_and_segment_agree_for_an_opaque_single_surface(renderer):
    """For one opaque Gaussian seen at its centre the two forms nearly agree:
    with alpha clamped at 0.99 they differ by 0.01 B_inf (e^{-beta_B d} -
    e^{-beta_B z_far}), the water behind it that only the segment form adds
    (below 3e-3 for this medium)."""
    g, m, cam = scenes.tiny_scene(2)
    n = g.means.shape[0]
    g.means[:] = g.means[0]
    g.log_scales[:] = -1.0
    g.opacity_logits[:] = -30.0
    g.opacity_logits[0] = 30.0
    params = R.params_to_device(g)
    med = medium_tensor(m)
    st = renderer.state()
    a = renderer.forward(st, params, med, cam, pixel=True)[0].cpu().numpy()
    b = renderer.forward(renderer.state(), params, med, cam)[0].cpu().numpy()
    fx, fy = cam.fx * g.means[0, 0] / g.means[0, 2] + cam.cx, cam.fy * g.means[0, 1] / g.means[0, 2] + cam.cy
    ix, iy = int(fx), int(fy)
    assert n > 1 and np.allclose(a[:, iy, ix], b[:, iy, ix], rtol=0, atol=4e-3)


def test_fused_pixel_step_equals_backward_then_adam(renderer):
    """The fused pixel-form training step updates every parameter as the
    pixel-form backward followed by the multi-group Adam does, and reports
    the same medium gradient."""
    from paper_2411_19588_b300 import warmstart
    g, m, cam = _box_scene(85, 1500, 100, 75, 90.0, 3, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    lr = dict(warmstart.FIT_LR)
    G = torch.tensor(np.random.default_rng(2).standard_normal((3, cam.height, cam.width)) * 0.1, dtype=torch.float32,
                     device="cuda")
    names = R.PARAM_NAMES + ("medium",)
    out = []
    for fused in (True, False):
        params = R.params_to_device(g)
        med = medium_tensor(m)
        tens = dict(params)
        tens["medium"] = med
        mo = {k: torch.zeros_like(tens[k]) for k in names}
        ve = {k: torch.zeros_like(tens[k]) for k in names}
        st = renderer.state()
        renderer.forward(st, params, med, cam, pixel=True)
        gm = torch.zeros(9, device="cuda")
        if fused:
            renderer.backward_adam(st, params, med, cam, G, mo, ve, lr, 1, grad_medium=gm, pixel=True)
        else:
            grads = renderer.backward(st, params, med, cam, G, pixel=True)
            gm.copy_(grads["medium"])
            groups = [{"param": tens[k], "grad": grads[k], "m": mo[k], "v": ve[k], "lr": lr[k],
                       "clamp_min": 0.0 if k == "medium" else None} for k in names]
            R.adam_step(groups, 1)
        torch.cuda.synchronize()
        out.append(({k: tens[k].cpu().numpy() for k in names}, gm.cpu().numpy()))
    for k in names:
        np.testing.assert_allclose(out[0][0][k], out[1][0][k], rtol=1e-6, atol=1e-7, err_msg=k)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-6, atol=1e-6)


def test_fit_in_the_pixel_form_lowers_the_loss(renderer):
    from paper_2411_19588_b300 import warmstart
    g, med, _ = scenes.patch_scene(20_000, 9, (2.0, 10.0), 320, 214, 300.0)
    cams = scenes.arc_cameras(6, 9, width=320, height=214, fx=300.0)
    gt = R.params_to_device(g)
    m = torch.tensor(med.as_array(), device="cuda")
    tgt = [renderer.forward(renderer.state(), gt, m, c, pixel=True)[0].clone() for c in cams]
    start, _ = scenes.perturb(g, med, seed=10)
    fit = warmstart.Fit(renderer, R.params_to_device(start), warmstart.DEFAULT_MEDIUM, cams, tgt, pixel=True)
    first = fit.psnr(range(6))
    for _ in range(60):
        fit.step()
    renderer.sync_status()
    assert fit.psnr(range(6)) > first + 1.0
