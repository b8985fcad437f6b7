"""The batched form (persistent blend over a (view, tile) queue, no host
synchronisation) against the plain per-view path, and under a CUDA graph."""
import numpy as np
import pytest
import torch

from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

pytestmark = pytest.mark.gpu


def _uneven_views(n_views, seed):
    cams = scenes.arc_cameras(n_views, seed, centroid=(0.0, 0.0, 4.5), radius=4.5, arc_len=3.0, width=128, height=96,
                              fx=120.0)
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        w = int(rng.integers(3, 12)) * 16 + int(rng.integers(0, 16))
        h = int(round(w / rng.uniform(4 / 3, 3 / 2)))
        f = 0.9375 * w
        out.append(scenes.Camera(w, h, f, f, w / 2, h / 2, c.world_to_cam, 0.2, 20.0))
    return out


@pytest.fixture(scope="module")
def scene(cuda_lib):
    g, m, _ = scenes.patch_scene(60_000, 21, (2.0, 7.0), 160, 120, 150.0)
    return R.params_to_device(g), torch.tensor(m.as_array(), device="cuda"), _uneven_views(5, 21)


@pytest.mark.parametrize("tile,batch", [((16, 16), 128), ((8, 32), 64), ((32, 8), 256), ((16, 16), 256)])
def test_batch_forward_equals_plain_renders(scene, tile, batch):
    params, med, cams = scene
    r = R.Renderer(tile=tile, batch=batch)
    b = R.Batch(r, cams)
    b.calibrate(params, med)
    imgs = [t.clone() for t in b.forward(params, med)]
    r.sync_status()
    plain = R.Renderer(tile=tile, batch=128)
    for v, cam in enumerate(cams):
        ref, _, _ = plain.render(params, med, cam)
        # same per-pixel arithmetic in the same order: bit-identical
        assert torch.equal(imgs[v], ref), (v, (imgs[v] - ref).abs().max().item())
    em, cap = b.pair_counts()
    assert all(e <= c for e, c in zip(em, cap))


def test_batch_backward_is_sum_of_view_gradients(scene):
    params, med, cams = scene
    r = R.Renderer()
    b = R.Batch(r, cams)
    b.calibrate(params, med)
    b.forward(params, med)
    rng = np.random.default_rng(3)
    ups = [torch.tensor(rng.standard_normal((3, c.height, c.width)), dtype=torch.float32, device="cuda") for c in cams]
    got = {k: v.clone() for k, v in b.backward(params, med, ups).items()}
    ref = None
    for cam, up in zip(cams, ups):
        st = r.state()
        r.forward(st, params, med, cam)
        gv = r.backward(st, params, med, cam, up)
        ref = {k: v.clone() for k, v in gv.items()} if ref is None else {k: ref[k] + gv[k] for k in ref}
    torch.cuda.synchronize()
    for k in ref:
        scale = ref[k].abs().max().item()
        torch.testing.assert_close(got[k], ref[k], rtol=1e-4, atol=1e-5 * scale)


def test_batch_under_cuda_graph_matches_eager(scene):
    params, med, cams = scene
    r = R.Renderer()
    b = R.Batch(r, cams)
    b.calibrate(params, med)
    rng = np.random.default_rng(4)
    ups = [torch.tensor(rng.standard_normal((3, c.height, c.width)), dtype=torch.float32, device="cuda") for c in cams]
    grads = {k: torch.zeros_like(params[k]) for k in R.PARAM_NAMES}
    grads["medium"] = torch.zeros_like(med)
    b.forward(params, med)
    b.backward(params, med, ups, grads)
    torch.cuda.synchronize()
    eager_img = [t.clone() for t in b.images]
    eager_g = {k: v.clone() for k, v in grads.items()}
    for v in grads.values():
        v.zero_()
    for t in b.images:
        t.zero_()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            b.forward(params, med)
            b.backward(params, med, ups, grads)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    r.sync_status()
    for a, e in zip(b.images, eager_img):
        assert torch.equal(a, e)
    for k in grads:
        torch.testing.assert_close(grads[k], eager_g[k], rtol=1e-4, atol=1e-5 * eager_g[k].abs().max().item())


def test_capacity_overflow_is_reported_not_faulted(scene):
    params, med, cams = scene
    r = R.Renderer()
    b = R.Batch(r, cams)
    b.calibrate(params, med, headroom=0.05)  # far too small on purpose
    b.forward(params, med)
    with pytest.raises(_abi.SplashError) as ei:
        r.sync_status()
    assert ei.value.status == _abi.ERR_CAPACITY
    # the context is intact: a fresh calibration renders correctly
    b.calibrate(params, med, headroom=1.25)
    imgs = b.forward(params, med)
    r.sync_status()
    ref, _, _ = r.render(params, med, cams[0])
    assert torch.equal(imgs[0], ref)


@pytest.mark.parametrize("batch", [64, 256])
def test_staging_batch_size_does_not_change_images(cuda_lib, batch):
    g, m, cam = scenes.tiny_scene(0)
    params = R.params_to_device(g)
    med = torch.tensor(m.as_array(), device="cuda")
    a, _, _ = R.Renderer(batch=128).render(params, med, cam)
    b, _, _ = R.Renderer(batch=batch).render(params, med, cam)
    assert torch.equal(a, b)


def test_batch_with_two_pass_tile_sorts_and_odd_gaussian_count(cuda_lib):
    """Views large enough that the tile sort takes two passes (>= 257 tiles),
    and a Gaussian count that is not a multiple of 4 (per-view slices of the
    key buffers then start at arbitrary offsets)."""
    g, m, _ = scenes.patch_scene(30_001, 23, (2.0, 7.0), 400, 300, 375.0)
    params = R.params_to_device(g)
    med = torch.tensor(m.as_array(), device="cuda")
    base = scenes.arc_cameras(3, 23, centroid=(0.0, 0.0, 4.5), radius=4.5, arc_len=2.0, width=400, height=300, fx=375.0)
    sizes = [(400, 300), (320, 240), (250, 200)]
    cams = [scenes.Camera(w, h, 0.9375 * w, 0.9375 * w, w / 2, h / 2, c.world_to_cam, 0.2, 20.0)
            for (w, h), c in zip(sizes, base)]
    r = R.Renderer()
    b = R.Batch(r, cams)
    b.calibrate(params, med)
    imgs = [t.clone() for t in b.forward(params, med)]
    ups = [torch.ones_like(t) * 1e-2 for t in imgs]
    got = {k: v.clone() for k, v in b.backward(params, med, ups).items()}
    r.sync_status()
    ref_g = None
    for v, cam in enumerate(cams):
        st = r.state()
        ref, _, _ = r.forward(st, params, med, cam)
        assert torch.equal(imgs[v], ref)
        gv = r.backward(st, params, med, cam, ups[v])
        ref_g = {k: x.clone() for k, x in gv.items()} if ref_g is None else {k: ref_g[k] + gv[k] for k in ref_g}
    for k in ref_g:
        torch.testing.assert_close(got[k], ref_g[k], rtol=1e-4, atol=1e-5 * ref_g[k].abs().max().item())
