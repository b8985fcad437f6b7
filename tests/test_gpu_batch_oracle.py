"""The batched form (one persistent blend launch over every (view, tile) of
a batch of uneven views, Sec. III-A tiles) against the FP64 oracle, view by
view, with the comparison protocol of the plain renderer; and the
autotuner's candidate table, cache and choice."""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_2411_19588_b300 import autotune
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import compare_forward, compare_grads, grads_to_numpy, upstream_keep
from test_gpu_forward import _box_scene

pytestmark = pytest.mark.gpu


def _ragged_views(n, seed):
    """n cameras around a box scene, widths 40-180 px, none a multiple of 16."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        w = int(rng.integers(40, 180))
        w += (w % 16 == 0)
        h = int(rng.integers(30, 140))
        h += (h % 16 == 0)
        f = 0.9 * w
        eye = rng.normal(0, 0.3, 3) + np.array([0.0, 0.0, -0.3])
        target = np.array([0.0, 0.0, 4.0]) + rng.normal(0, 0.2, 3)
        c = scenes.look_at(eye, target, w, h, f, f)
        cams.append(c)
    return cams


def _batch_forward(r, params, med, cams):
    b = R.Batch(r, cams)
    b.calibrate(params, med)
    depths = [torch.empty((c.height, c.width), device="cuda") for c in cams]
    d01 = [torch.empty((c.height, c.width), device="cuda") for c in cams]
    imgs = b.forward(params, med, depths=depths, depth01s=d01)
    torch.cuda.synchronize()
    r.sync_status()
    out = [{"image": i.cpu().numpy().astype(np.float64), "depth": d.cpu().numpy().astype(np.float64),
            "depth01": z.cpu().numpy().astype(np.float64)} for i, d, z in zip(imgs, depths, d01)]
    return b, out


@pytest.mark.parametrize("tile,batch", [((16, 16), 64), ((8, 32), 128), ((32, 8), 256)])
def test_batched_views_match_oracle(cuda_lib, tile, batch):
    """Nine ragged views in one batch: every view's image and depths against
    the oracle at every pixel, and the batch's summed gradient against the
    sum of the oracle's per-view adjoints (each on the branches the view's
    forward matched)."""
    g, m, _ = _box_scene(101, 2500, 100, 75, 90.0, 3)
    cams = _ragged_views(9, 101)
    params = R.params_to_device(g)
    med = torch.tensor(m.as_array(), dtype=torch.float32, device="cuda")
    r = R.Renderer(tile=tile, batch=batch)
    b, outs = _batch_forward(r, params, med, cams)
    rng = np.random.default_rng(7)
    ups, ref = [], None
    for v, (cam, out) in enumerate(zip(cams, outs)):
        ora = oracle.render(g, m, cam)
        fwd = compare_forward(out, ora, label=f"batch {tile[0]}x{tile[1]} view {v} {cam.width}x{cam.height}",
                              scene=(g, m, cam))
        G = np.float64(np.float32(rng.standard_normal((3, cam.height, cam.width)) * upstream_keep(ora, fwd)))
        ups.append(torch.tensor(G, dtype=torch.float32, device="cuda"))
        gv = oracle.backward(g, m, cam, G, branch=fwd["branch"])
        ref = gv if ref is None else {k: ref[k] + gv[k] for k in ref}
    got = grads_to_numpy(b.backward(params, med, ups))
    r.sync_status()
    print(tile, compare_grads(got, ref, f"batch {tile[0]}x{tile[1]}"))


def test_batched_full_workload_sampled(cuda_lib):
    """The batched workload at its own shape: 64 views from 640x480 to
    1920x1280 over the 1.5M-Gaussian scene, one persistent launch each way.
    Six sampled pixels per view against the oracle forward; backward, an
    upstream gradient non-zero at those pixels only, summed over the views,
    against the sum of the oracle's adjoints at the same pixels."""
    g, m, _ = scenes.full_scene()
    cams = scenes.uneven_cameras(64, 4)
    assert min(c.width for c in cams) >= 640 and max(c.width for c in cams) <= 1920
    params = R.params_to_device(g)
    med = torch.tensor(m.as_array(), dtype=torch.float32, device="cuda")
    r = R.Renderer()
    b, outs = _batch_forward(r, params, med, cams)
    rng = np.random.default_rng(11)
    ups, ref = [], None
    for v, (cam, out) in enumerate(zip(cams, outs)):
        pix = rng.choice(cam.width * cam.height, 6, replace=False)
        ora = oracle.render(g, m, cam, pix=pix)
        fwd = compare_forward(out, ora, pix=pix, label=f"batch full view {v}", scene=(g, m, cam))
        keep = upstream_keep(ora, fwd)
        Gs = np.float64(np.float32(rng.standard_normal((3, pix.size)))) * keep
        G = np.zeros((3, cam.height * cam.width), np.float32)
        G[:, pix] = Gs
        ups.append(torch.tensor(G.reshape(3, cam.height, cam.width), device="cuda"))
        gv = oracle.backward(g, m, cam, Gs, pix=pix, branch=fwd["branch"])
        ref = gv if ref is None else {k: ref[k] + gv[k] for k in ref}
    got = grads_to_numpy(b.backward(params, med, ups))
    r.sync_status()
    assert np.abs(ref["means"]).sum() > 0
    print("batch full", compare_grads(got, ref, "batch full"))
    assert all(np.isfinite(o["image"]).all() for o in outs)


def test_autotuner_table_cache_and_choice(cuda_lib, tmp_path):
    """Nine candidates (three tile shapes x three staging batches) are timed;
    the winner is written to the cache under the batch's key and read back
    without timing; a renderer built with the chosen configuration renders
    the batch exactly as 16x16 / 128 does (membership is per pixel, so every
    configuration composites the same lists in the same order)."""
    g, m, _ = _box_scene(111, 3000, 120, 90, 100.0, 3)
    cams = _ragged_views(4, 111)
    params = R.params_to_device(g)
    params["sh_degree"] = g.sh_degree
    med = torch.tensor(m.as_array(), dtype=torch.float32, device="cuda")
    path = str(tmp_path / "tune.json")
    first = autotune.autotune(params, med, cams, reps=1, path=path)
    assert not first["cached"]
    assert len(first["table"]) == 9
    assert set(first["table"]) == {f"{t[0]}x{t[1]}/{nb}" for t in autotune.TILES for nb in autotune.BATCHES}
    assert all(v > 0 for v in first["table"].values())
    assert first["ms"] == min(first["table"].values())
    assert f"{first['tile'][0]}x{first['tile'][1]}/{first['batch']}" == min(first["table"], key=first["table"].get)
    with open(path) as f:
        disk = json.load(f)
    key = autotune.cache_key(params, cams)
    assert list(disk) == [key] and disk[key]["batch"] == first["batch"]
    again = autotune.autotune(params, med, cams, reps=1, path=path)
    assert again["cached"] and again["tile"] == first["tile"] and again["batch"] == first["batch"]
    # another view set is another key
    other = autotune.cache_key(params, cams[:3])
    assert other != key
    # the chosen configuration renders the batch bit for bit as the default one
    _, a = _batch_forward(R.Renderer(tile=first["tile"], batch=first["batch"]), params, med, cams)
    _, b = _batch_forward(R.Renderer(tile=(16, 16), batch=128), params, med, cams)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["image"], y["image"])
        np.testing.assert_array_equal(x["depth"], y["depth"])
