"""Error paths on the GPU: every failure is made on the host (bad arguments,
a partition that never reports) and must come back as a status code with
the context still usable. Nothing here faults, traps or hangs the GPU: the
device-side wait that is made to run out is bounded by spin_limit."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import render as R
from paper_2411_19588_b300 import scenes

from parity import gpu_forward

pytestmark = pytest.mark.gpu


def test_invalid_arguments_are_rejected(cuda_lib):
    L = _abi.lib()
    h = ctypes.c_void_p()
    assert L.splash_create(ctypes.byref(_abi.Options(12, 12, 0, 0, 0)), ctypes.byref(h)) == _abi.ERR_INVALID_ARG
    assert L.splash_create(ctypes.byref(_abi.Options(16, 16, 0, 0, 96)), ctypes.byref(h)) == _abi.ERR_INVALID_ARG
    r = R.Renderer()
    st = r.state()
    g, m, cam = scenes.tiny_scene(0)
    params = R.params_to_device(g)
    med = torch.tensor(m.as_array(), device="cuda")
    gs = R.gaussians_struct(params)
    c = R.camera_struct(cam)
    img = torch.empty((3, cam.height, cam.width), device="cuda")
    s = R._stream()
    # sh degree out of range
    gs.sh_degree = 4
    assert L.splash_render_forward(r._ctx, st.handle, ctypes.byref(gs), med.data_ptr(), ctypes.byref(c), img.data_ptr(),
                                   None, None, s) == _abi.ERR_INVALID_ARG
    gs.sh_degree = 0
    # zero-size image, null image, null medium
    c.width = 0
    assert L.splash_render_forward(r._ctx, st.handle, ctypes.byref(gs), med.data_ptr(), ctypes.byref(c), img.data_ptr(),
                                   None, None, s) == _abi.ERR_INVALID_ARG
    c.width = cam.width
    assert L.splash_render_forward(r._ctx, st.handle, ctypes.byref(gs), med.data_ptr(), ctypes.byref(c), None, None, None,
                                   s) == _abi.ERR_INVALID_ARG
    assert L.splash_render_forward(r._ctx, st.handle, ctypes.byref(gs), None, ctypes.byref(c), img.data_ptr(), None, None,
                                   s) == _abi.ERR_INVALID_ARG
    # backward before any forward on a fresh state
    st2 = r.state()
    gr = _abi.Grads()
    assert L.splash_render_backward(r._ctx, st2.handle, ctypes.byref(gs), med.data_ptr(), ctypes.byref(c),
                                    img.data_ptr(), None, None, ctypes.byref(gr), s) == _abi.ERR_STATE
    assert b"forward" in L.splash_last_error()
    # the context still renders correctly afterwards
    out = gpu_forward(r, g, m, cam)
    assert np.isfinite(out["image"]).all()


def test_nan_parameters_are_culled(cuda_lib):
    """A Gaussian with a NaN in any parameter group touches no tile, and the
    rest of the scene renders exactly as the scene without it: same image
    and depth bit for bit (their relative depth order, ties included, is
    unchanged by removing others)."""
    r = R.Renderer()
    g, m, cam = scenes.tiny_scene(0)
    g = g.copy()
    bad = np.zeros(g.n, bool)
    for arr, start, step in ((g.means, 0, 7), (g.log_scales, 1, 11), (g.quats, 2, 13), (g.opacity_logits, 3, 17),
                             (g.sh, 4, 19)):
        arr[start::step] = np.nan
        bad[start::step] = True
    out = gpu_forward(r, g, m, cam)
    r.sync_status()
    tt = r.state_array(out["state"], "tiles_touched").cpu().numpy().view(np.uint32)
    assert (tt[bad] == 0).all()
    assert (tt[~bad] > 0).sum() > 100
    keep = np.flatnonzero(~bad)
    sub = scenes.Gaussians(*(np.ascontiguousarray(a[keep]) for a in (g.means, g.log_scales, g.quats, g.opacity_logits,
                                                                     g.sh)), g.sh_degree)
    ref = gpu_forward(R.Renderer(), sub, m, cam)
    np.testing.assert_array_equal(out["image"], ref["image"])
    np.testing.assert_array_equal(out["depth"], ref["depth"])
    assert np.isfinite(out["image"]).all()


def test_stalled_lookback_reports_timeout_and_context_survives(cuda_lib):
    """Partition 2 of every sort pass never publishes; partition 3's bounded
    wait runs out, the kernel sets the status word and returns, and the call
    reports SPLASH_ERR_TIMEOUT. The same process then renders correctly."""
    bad = R.Renderer(spin_limit=20000, test_stall_partition=2)
    st = bad.state()
    n = 5 * 4096 + 17
    keys = torch.randint(0, 1 << 20, (n,), dtype=torch.int32, device="cuda")
    with pytest.raises(_abi.SplashError) as ei:
        bad.sort_pairs(st, keys, None, 20)
        bad.sync_status()
    assert ei.value.status == _abi.ERR_TIMEOUT
    bad.sync_status()  # the status word was cleared
    good = R.Renderer()
    ko, vo = good.sort_pairs(good.state(), keys, None, 20)
    good.sync_status()
    ref = np.argsort(keys.cpu().numpy().astype(np.int64), kind="stable")
    np.testing.assert_array_equal(vo.cpu().numpy(), ref)


@pytest.mark.parametrize("n", [120_000, 500_000])
def test_pair_count_beyond_capacity_is_reported(cuda_lib, n):
    """Screen-filling Gaussians at 1920x1280 (9,600 tiles each): 120k give
    about 1.15e9 pairs (past the 2^30 limit), 500k about 4.8e9 (past 2^32,
    where a 32-bit sum would wrap to a small count). The pair count is summed
    in 64 bits, so both are refused with SPLASH_ERR_CAPACITY before any pair
    buffer is sized from it, and the context renders correctly afterwards."""
    r = R.Renderer()
    cam = scenes.Camera(1920, 1280, 1800.0, 1800.0, 960.0, 640.0, np.concatenate([np.eye(3), np.zeros((3, 1))], 1),
                        0.2, 20.0)
    rng = np.random.default_rng(n)
    g = scenes.Gaussians(np.float32(np.c_[rng.uniform(-0.1, 0.1, (n, 2)), rng.uniform(3.0, 4.0, n)]),
                         np.full((n, 3), 2.0, np.float32), np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                         np.full(n, 2.0, np.float32), np.zeros((n, 1, 3), np.float32), 0)
    med = scenes.Medium(np.float32([0.1] * 3), np.float32([0.1] * 3), np.float32([0.1] * 3))
    with pytest.raises(_abi.SplashError) as ei:
        gpu_forward(r, g, med, cam)
    assert ei.value.status == _abi.ERR_CAPACITY
    assert b"2^30" in _abi.lib().splash_last_error()
    g2, m2, cam2 = scenes.tiny_scene(0)
    out = gpu_forward(r, g2, m2, cam2)
    assert np.isfinite(out["image"]).all()
