"""Backward parity of the CUDA rasterizer against the oracle's FP64 adjoint
(itself pinned by FP64 central differences), taken on the branch of each
pixel's near decisions that the GPU's forward matched. Upstream gradients
are zeroed, on both sides, only at pixels two branches match and at pixels
near a gradient kink (counted in the session's parity summary)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import compare_forward, compare_grads, gpu_forward, grads_to_numpy, medium_tensor, upstream_keep
from test_gpu_forward import _box_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


def _upstream(rng, keep, H, W, depth=True):
    G = rng.standard_normal((3, H, W)) * keep
    Gz = rng.standard_normal((H, W)) * 0.05 * keep if depth else np.zeros((H, W))
    G01 = rng.standard_normal((H, W)) * 0.3 * keep if depth else np.zeros((H, W))
    return G, Gz, G01, keep


def _run(renderer, g, m, cam, seed, depth=True, label="bwd"):
    gpu = gpu_forward(renderer, g, m, cam)
    ora = oracle.render(g, m, cam)
    fwd = compare_forward(gpu, ora, label=label, scene=(g, m, cam))
    rng = np.random.default_rng(seed)
    G, Gz, G01, keep = _upstream(rng, upstream_keep(ora, fwd), cam.height, cam.width, depth)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    # the oracle sees exactly the FP32 upstream values the GPU sees
    G, Gz, G01 = (np.float64(np.float32(a)) for a in (G, Gz, G01))
    grads = renderer.backward(gpu["state"], gpu["params"], gpu["medium"], cam, t(G), t(Gz), t(G01))
    torch.cuda.synchronize()
    ref = oracle.backward(g, m, cam, G, Gz, G01, branch=fwd["branch"])
    return grads_to_numpy(grads), ref, keep


def test_tiny_scene_gradients(renderer):
    g, m, cam = scenes.tiny_scene(0)
    got, ref, keep = _run(renderer, g, m, cam, 1, label="bwd tiny")
    print("tiny", compare_grads(got, ref, "tiny"), "kept", keep.mean())


@pytest.mark.parametrize("seed,W,H,deg", [(51, 100, 75, 3), (52, 61, 47, 1)])
def test_ragged_gradients(renderer, seed, W, H, deg):
    g, m, cam = _box_scene(seed, 1500, W, H, 0.9 * W, deg, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    got, ref, _ = _run(renderer, g, m, cam, seed, label=f"bwd ragged{W}x{H}")
    print((W, H), compare_grads(got, ref, f"ragged{W}x{H}"))


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_other_tile_shapes_gradients(cuda_lib, tile):
    """The plain backward with the autotuner's other tile shapes (64
    threads of 4 pixels each, 2 or 8 threads per tile row) on a ragged image
    with and without the depth terms."""
    r = R.Renderer(tile=tile)
    g, m, cam = _box_scene(71, 1500, 100, 75, 90.0, 3, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    for depth in (True, False):
        got, ref, _ = _run(r, g, m, cam, 71, depth, label=f"bwd tile{tile[0]}x{tile[1]} depth={depth}")
        print(tile, depth, compare_grads(got, ref, f"tile{tile[0]}x{tile[1]}"))


def test_dense_overlap_gradients(renderer):
    """Long per-pixel lists: checks the back-to-front recomputation of T
    from the stored final transmittance."""
    g, m, cam = _box_scene(61, 2500, 80, 60, 70.0, 3, log_scale=-1.7)
    got, ref, _ = _run(renderer, g, m, cam, 61, label="bwd dense")
    print("dense", compare_grads(got, ref, "dense"))


def test_image_only_upstream(renderer):
    g, m, cam = _box_scene(71, 1200, 64, 48, 60.0, 2)
    got, ref, _ = _run(renderer, g, m, cam, 71, depth=False, label="bwd image-only")
    compare_grads(got, ref, "image-only")


def test_full_scene_sparse_upstream(renderer):
    """1.5M Gaussians at 1920x1280: an upstream gradient that is non-zero at
    200 sampled pixels only, so the oracle's exact gradient needs just those
    pixels; every parameter gradient is compared."""
    g, m, cam = scenes.full_scene()
    gpu = gpu_forward(renderer, g, m, cam)
    rng = np.random.default_rng(8)
    pix = rng.choice(cam.width * cam.height, 200, replace=False)
    ora = oracle.render(g, m, cam, pix=pix)
    fwd = compare_forward(gpu, ora, pix=pix, label="bwd full", scene=(g, m, cam))
    keep = upstream_keep(ora, fwd)
    pix, branch = pix[keep], fwd["branch"][keep]
    H, W = cam.height, cam.width
    Gs = np.float64(np.float32(rng.standard_normal((3, pix.size))))
    Gzs = np.float64(np.float32(rng.standard_normal(pix.size) * 0.05))
    G01s = np.float64(np.float32(rng.standard_normal(pix.size) * 0.3))
    G = np.zeros((3, H * W), np.float32)
    Gz = np.zeros(H * W, np.float32)
    G01 = np.zeros(H * W, np.float32)
    G[:, pix], Gz[pix], G01[pix] = Gs, Gzs, G01s
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    grads = renderer.backward(gpu["state"], gpu["params"], gpu["medium"], cam, t(G.reshape(3, H, W)),
                              t(Gz.reshape(H, W)), t(G01.reshape(H, W)))
    torch.cuda.synchronize()
    ref = oracle.backward(g, m, cam, Gs, Gzs, G01s, pix=pix, branch=branch)
    assert np.abs(ref["means"]).sum() > 0
    print("full", compare_grads(grads_to_numpy(grads), ref, "full-sparse"))


def test_autograd_function_matches_direct_backward(renderer):
    g, m, cam = _box_scene(81, 800, 48, 40, 45.0, 3)
    params = R.params_to_device(g)
    leaves = {k: params[k].clone().requires_grad_(True) for k in R.PARAM_NAMES}
    med = medium_tensor(m).requires_grad_(True)
    p2 = dict(leaves, sh_degree=g.sh_degree)
    img, depth, depth01 = R.render(p2, med, cam, renderer)
    rng = np.random.default_rng(3)
    G = torch.tensor(rng.standard_normal((3, cam.height, cam.width)), dtype=torch.float32, device="cuda")
    Gz = torch.tensor(rng.standard_normal((cam.height, cam.width)), dtype=torch.float32, device="cuda")
    ((img * G).sum() + (depth * Gz).sum()).backward()
    gpu = gpu_forward(renderer, g, m, cam)
    direct = renderer.backward(gpu["state"], gpu["params"], gpu["medium"], cam, G, Gz, None)
    for k in R.PARAM_NAMES:
        torch.testing.assert_close(leaves[k].grad, direct[k], rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(med.grad, direct["medium"], rtol=1e-5, atol=1e-6)
