"""Forward parity of the CUDA rasterizer against the FP64 oracle, plus the
bit-exact checks of binning and sorting. Everything goes through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import compare_forward, gpu_forward, medium_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer(cuda_lib):
    return R.Renderer()


def _box_scene(seed, n, W, H, f, deg, eye=(0.0, 0.0, 0.0), target=(0.0, 0.0, 3.0), log_scale=-2.6):
    rng = np.random.default_rng(seed)
    cam = scenes.look_at(eye, target, W, H, f, f)
    c = cam.center + 3.5 * (np.asarray(target) - np.asarray(eye)) / np.linalg.norm(np.asarray(target) - np.asarray(eye))
    means = c + np.c_[rng.uniform(-1.5, 1.5, (n, 2)), rng.uniform(-2.5, 2.5, n)]
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.1, (n, K, 3))
    sh[:, 0, :] = (rng.uniform(0, 1, (n, 3)) - 0.5) / 0.28209479177387814
    g = scenes.Gaussians(*(np.ascontiguousarray(a, np.float32) for a in (
        means, rng.normal(log_scale, 0.5, (n, 3)), rng.standard_normal((n, 4)), rng.normal(0.5, 1.0, n), sh)), deg)
    return g, scenes.random_medium(rng), cam


def test_tiny_scene_matches_oracle(renderer):
    """1,000 Gaussians, 128x96, SH degree 0 (the small workload)."""
    g, m, cam = scenes.tiny_scene(0)
    gpu = gpu_forward(renderer, g, m, cam)
    ora = oracle.render(g, m, cam)
    stats = compare_forward(gpu, ora, label="tiny", scene=(g, m, cam))
    print("tiny", stats)


@pytest.mark.parametrize("seed,W,H,deg", [(11, 100, 75, 3), (12, 37, 141, 1), (13, 257, 19, 2)])
def test_ragged_images_match_oracle(renderer, seed, W, H, deg):
    """Sizes that leave partial tiles on both axes; rotated camera; SH 1-3."""
    g, m, cam = _box_scene(seed, 2500, W, H, 0.9 * W, deg, eye=(0.3, -0.2, -0.4), target=(0.1, 0.05, 4.0))
    gpu = gpu_forward(renderer, g, m, cam)
    ora = oracle.render(g, m, cam)
    print((W, H), compare_forward(gpu, ora, label=f"ragged{W}x{H}", scene=(g, m, cam)))


def test_dense_overlap_matches_oracle(renderer):
    """Large, strongly overlapping Gaussians: long lists and early stops."""
    g, m, cam = _box_scene(21, 3000, 96, 64, 80.0, 3, log_scale=-1.6)
    gpu = gpu_forward(renderer, g, m, cam)
    ora = oracle.render(g, m, cam)
    assert ora["n_contrib"].max() >= 20
    print("dense", compare_forward(gpu, ora, label="dense", scene=(g, m, cam)))


@pytest.mark.parametrize("tile", [(8, 32), (32, 8)])
def test_tile_shapes_give_identical_images(cuda_lib, tile):
    """Membership is decided per pixel (3-sigma ellipse), so every tile
    shape composites the same Gaussians in the same order: bit-identical."""
    g, m, cam = _box_scene(31, 3000, 150, 110, 120.0, 3)
    a = gpu_forward(R.Renderer(tile=(16, 16)), g, m, cam)
    b = gpu_forward(R.Renderer(tile=tile), g, m, cam)
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["depth"], b["depth"])


def test_empty_and_culled_scenes(renderer):
    med = scenes.Medium(np.array([0.4, 0.2, 0.1], np.float32), np.array([0.3, 0.25, 0.2], np.float32),
                        np.array([0.05, 0.2, 0.3], np.float32))
    cam = scenes.Camera(70, 50, 60.0, 60.0, 35.0, 25.0, np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 0.2, 20.0)
    expect = med.b_inf.astype(np.float64) * (1 - np.exp(-med.beta_b.astype(np.float64) * 20.0))
    empty = scenes.Gaussians(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32),
                             np.zeros(0, np.float32), np.zeros((0, 1, 3), np.float32), 0)
    rng = np.random.default_rng(3)
    behind = scenes.Gaussians(np.c_[rng.uniform(-1, 1, (50, 2)), rng.uniform(-3, 0.1, 50)].astype(np.float32),
                              np.full((50, 3), -1.0, np.float32), np.tile(np.float32([1, 0, 0, 0]), (50, 1)),
                              np.full(50, 3.0, np.float32), np.zeros((50, 1, 3), np.float32), 0)
    for g in (empty, behind):
        out = gpu_forward(renderer, g, med, cam)
        np.testing.assert_allclose(out["image"], np.broadcast_to(expect[:, None, None], out["image"].shape), atol=1e-6)
        np.testing.assert_allclose(out["depth"], 20.0)


def test_culled_padding_keeps_the_image(renderer):
    """4.4M Gaussians behind the camera added to a 3,000-Gaussian scene: they are
    culled and list no tiles, so the image and depth stay bit for bit the same;
    with more than 1,024 chunks of 4,096 depth-ordered Gaussians the count scan
    takes its separate top-level pass."""
    g, m, cam = _box_scene(91, 3000, 160, 120, 140.0, 1)
    extra = 4_400_000
    rng = np.random.default_rng(92)
    pad = lambda a, b: np.ascontiguousarray(np.concatenate([a, b]), np.float32)
    big = scenes.Gaussians(
        pad(g.means, np.c_[rng.uniform(-2, 2, (extra, 2)), rng.uniform(-5.0, -0.5, extra)]),
        pad(g.log_scales, np.full((extra, 3), -2.0)), pad(g.quats, np.tile([1.0, 0, 0, 0], (extra, 1))),
        pad(g.opacity_logits, np.full(extra, 2.0)), pad(g.sh, np.zeros((extra,) + g.sh.shape[1:])), g.sh_degree)
    a = gpu_forward(renderer, g, m, cam)
    b = gpu_forward(renderer, big, m, cam)
    assert big.n > 1024 * 4096
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["depth"], b["depth"])


def test_one_pixel_image(renderer):
    g, m, _ = scenes.tiny_scene(0)
    cam = scenes.Camera(1, 1, 120.0, 120.0, 0.5, 0.5, np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 0.2, 20.0)
    compare_forward(gpu_forward(renderer, g, m, cam), oracle.render(g, m, cam), label="1x1", scene=(g, m, cam))


@pytest.mark.parametrize("n,z_step,W,H,f,log_scale", [
    (4000, 0.0, 203, 157, 150.0, -2.2), (5 * 5120 + 77, 0.25, 203, 157, 150.0, -2.2),
    # more super-tiles, partial ones on both edges
    (6000, 0.0, 1000, 700, 900.0, -3.6),
    # 24 x 32 super-tiles: their sort takes two passes
    (4000, 0.0, 3000, 2000, 2700.0, -4.5),
    # a tile grid whose count array does not fit in shared memory: the pairs are sorted by tile instead
    (4000, 0.0, 4200, 4200, 3780.0, -4.5)])
def test_binning_and_sort_bit_exact(renderer, n, z_step, W, H, f, log_scale):
    """Each Gaussian is listed in the tiles of its rectangle; the lists equal
    a CPU stable sort of 64-bit (tile << 32 | depth bits) keys emitted in
    Gaussian-index order; ranges equal a linear scan. The second case spans
    several depth-sort partitions with a ragged last one, and its depths sit
    on planes z_step apart (the camera looks down +z from the origin), so that
    thousands of Gaussians share one depth key and their order within a tile
    is decided by the sorts' stability alone. The other cases take the
    two-level binning over many super-tiles (8 x 4 tiles each), with one and
    with two sort passes, and the sort-by-tile path of very large images."""
    g, m, cam = _box_scene(41, n, W, H, f, 3, log_scale=log_scale)
    if z_step:
        g.means[:, 2] = np.round(g.means[:, 2] / z_step) * z_step
    out = gpu_forward(renderer, g, m, cam)
    st = out["state"]
    info = renderer.info(st)
    dk = renderer.state_array(st, "depth_keys").cpu().numpy().view(np.uint32)
    tt = renderer.state_array(st, "tiles_touched").cpu().numpy().view(np.uint32)
    rects = renderer.state_array(st, "rects").cpu().numpy().view(np.uint32)
    tids = renderer.state_array(st, "tile_ids").cpu().numpy().view(np.uint32)
    gids = renderer.state_array(st, "gauss_ids").cpu().numpy().view(np.uint32)
    ranges = renderer.state_array(st, "ranges").cpu().numpy().view(np.uint32)
    tx = info["tiles_x"]
    keys, ids = [], []
    for i in range(g.n):
        if tt[i] == 0:
            continue
        x0, x1, y0, y1 = rects[i, 0] & 0xFFFF, rects[i, 0] >> 16, rects[i, 1] & 0xFFFF, rects[i, 1] >> 16
        assert tt[i] == (x1 - x0 + 1) * (y1 - y0 + 1)
        assert dk[i] != 0xFFFFFFFF
        for ty in range(y0, y1 + 1):
            for t in range(x0, x1 + 1):
                keys.append((np.uint64(ty * tx + t) << np.uint64(32)) | np.uint64(dk[i]))
                ids.append(i)
    keys = np.array(keys, np.uint64)
    ids = np.array(ids, np.uint32)
    if z_step:
        assert np.unique(dk[tt > 0]).size <= 25  # few distinct depth keys: many ties
    order = np.argsort(keys, kind="stable")
    assert info["n_keys"] == keys.size
    np.testing.assert_array_equal(tids, (keys[order] >> np.uint64(32)).astype(np.uint32))
    np.testing.assert_array_equal(gids, ids[order])
    # ranges: each tile's run in the sorted ids (an empty tile's is [s, s),
    # s the number of pairs of the tiles before it)
    ntiles = info["tiles_x"] * info["tiles_y"]
    tile_no = np.arange(ntiles)
    exp = np.stack([np.searchsorted(tids, tile_no, "left"), np.searchsorted(tids, tile_no, "right")], 1)
    np.testing.assert_array_equal(ranges, exp.astype(np.uint32))


@pytest.mark.parametrize("n,bits,distinct", [(1, 32, 10), (4095, 13, 50), (4097, 32, 1 << 30), (100_003, 14, 9600),
                                             (3_000_001, 32, 1 << 31), (1_234_567, 20, 300), (70_000, 0, 1),
                                             # 9-bit digit plans: 9, 9+8, 9+9+8, 9+9+9 bits
                                             (5_000, 9, 1 << 9), (300_001, 17, 1 << 17), (1_500_000, 26, 1 << 26),
                                             (1_000_003, 26, 5000), (70_001, 27, 1 << 32)])
def test_radix_sort_bit_exact(renderer, n, bits, distinct):
    """Stable sort on key bits [0, bits) against numpy's stable argsort (keys
    may carry bits above `bits`: they are ignored)."""
    rng = np.random.default_rng(n)
    keys = rng.integers(0, distinct, n, dtype=np.int64).astype(np.uint32)
    vals = rng.integers(0, 1 << 31, n, dtype=np.int64).astype(np.uint32)
    st = renderer.state()
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = renderer.sort_pairs(st, kt, vt, bits)
    renderer.sync_status()
    masked = keys & np.uint32((1 << bits) - 1) if bits < 32 else keys
    order = np.argsort(masked, kind="stable")
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
    # values default to the input positions
    _, io = renderer.sort_pairs(st, kt, None, bits)
    np.testing.assert_array_equal(io.cpu().numpy().view(np.uint32), order.astype(np.uint32))


def test_mid_scene_sampled_pixels(renderer):
    """300k-Gaussian surface-patch scene at 1280x854, SH degree 3: sampled
    pixels against the oracle computed pixel by pixel."""
    g, m, cam = scenes.mid_scene()
    gpu = gpu_forward(renderer, g, m, cam)
    rng = np.random.default_rng(5)
    pix = rng.choice(cam.width * cam.height, 400, replace=False)
    ora = oracle.render(g, m, cam, pix=pix)
    print("mid", compare_forward(gpu, ora, pix=pix, label="mid", scene=(g, m, cam)))


def test_full_scene_sampled_pixels(renderer):
    """1.5M Gaussians at 1920x1280 (the benchmark workload and launch
    configuration): sampled pixels against the oracle."""
    g, m, cam = scenes.full_scene()
    gpu = gpu_forward(renderer, g, m, cam)
    rng = np.random.default_rng(6)
    pix = rng.choice(cam.width * cam.height, 200, replace=False)
    ora = oracle.render(g, m, cam, pix=pix)
    print("full", compare_forward(gpu, ora, pix=pix, label="full", scene=(g, m, cam)))
    # every pixel is finite; the image stays in the physical range
    assert np.isfinite(gpu["image"]).all() and gpu["image"].min() >= -1e-6
