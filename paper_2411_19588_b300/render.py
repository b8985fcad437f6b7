"""Torch-facing API of the rasterizer: tensors in, tensors out, all work in
libsplash's kernels (argument marshalling only here).

    r = Renderer()                                   # tile 16x16
    img, depth, depth01 = r.render(params, medium, camera)
    img, depth, depth01 = render(params, medium, camera, renderer=r)  # autograd

``params`` holds CUDA float32 contiguous tensors ``means`` [n,3],
``log_scales`` [n,3], ``quats`` [n,4] (w,x,y,z), ``opacity_logits`` [n],
``sh`` [n,(deg+1)^2,3]; ``medium`` is a CUDA float32 [9] tensor
(beta_D[3], beta_B[3], B_inf[3]); ``camera`` is a ``scenes.Camera``.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _abi
from . import scenes

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def camera_struct(cam: scenes.Camera) -> _abi.Camera:
    c = _abi.Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    w2c = np.asarray(cam.world_to_cam, np.float32).reshape(12)
    for i in range(12):
        c.world_to_cam[i] = float(w2c[i])
    c.z_near, c.z_far = float(cam.z_near), float(cam.z_far)
    return c


def _check_tensor(t: torch.Tensor, name: str, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def params_to_device(g: scenes.Gaussians, device="cuda") -> dict:
    out = {k: torch.from_numpy(np.ascontiguousarray(getattr(g, k), np.float32)).to(device) for k in PARAM_NAMES}
    out["sh_degree"] = int(g.sh_degree)
    return out


def gaussians_struct(p: dict) -> _abi.Gaussians:
    n = p["means"].shape[0]
    deg = int(p["sh_degree"])
    K = (deg + 1) ** 2
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity_logits": (n,), "sh": (n, K, 3)}
    for k in PARAM_NAMES:
        _check_tensor(p[k], k, shapes[k])
    g = _abi.Gaussians()
    g.means, g.log_scales, g.quats = p["means"].data_ptr(), p["log_scales"].data_ptr(), p["quats"].data_ptr()
    g.opacity_logits, g.sh = p["opacity_logits"].data_ptr(), p["sh"].data_ptr()
    g.n, g.sh_degree = n, deg
    return g


class State:
    """A render workspace (device buffers grow on demand). Returned to its
    renderer's pool when garbage collected."""

    def __init__(self, renderer: "Renderer", handle: ctypes.c_void_p):
        self._renderer = renderer
        self.handle = handle
        self.shape = None

    def __del__(self):
        r = getattr(self, "_renderer", None)
        if r is not None and self.handle:
            r._release(self.handle)
            self.handle = None


class Renderer:
    """One library context (splash_create). tile: pixel tile (16, 16), (8, 32)
    or (32, 8); batch: Gaussians staged in shared memory per blend step, 64,
    128 or 256 for both passes, or 0 for the per-pass defaults (forward 64,
    backward 128); spin_limit: iterations before a device wait gives up (0:
    the library default); test_stall_partition: testing aid of the sort's
    bounded waits (0: off)."""

    def __init__(self, tile=(16, 16), spin_limit: int = 0, test_stall_partition: int = 0, batch: int = 0):
        L = _abi.lib()
        opt = _abi.Options(int(tile[0]), int(tile[1]), int(spin_limit), int(test_stall_partition), int(batch))
        h = ctypes.c_void_p()
        _abi.check(L.splash_create(ctypes.byref(opt), ctypes.byref(h)), "splash_create")
        self._ctx = h
        self._pool = []
        self.tile = tuple(tile)

    def close(self):
        L = _abi.lib()
        for h in self._pool:
            L.splash_state_destroy(h)
        self._pool = []
        if self._ctx:
            L.splash_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- states
    def state(self) -> State:
        if self._pool:
            return State(self, self._pool.pop())
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().splash_state_create(self._ctx, ctypes.byref(h)), "splash_state_create")
        return State(self, h)

    def _release(self, h):
        if self._ctx:
            self._pool.append(h)
        else:
            _abi.lib().splash_state_destroy(h)

    # -- render
    def forward(self, st: State, params: dict, medium: torch.Tensor, cam: scenes.Camera, image=None, depth=None,
                depth01=None, pixel: bool = False):
        """Render (image, depth, depth01). pixel=True: Eq. 5 applied per pixel
        with the Eq. 6 depth instead of per Gaussian and water segment."""
        _check_tensor(medium, "medium", (9,))
        H, W = cam.height, cam.width
        dev = medium.device
        image = torch.empty((3, H, W), device=dev, dtype=torch.float32) if image is None else image
        depth = torch.empty((H, W), device=dev, dtype=torch.float32) if depth is None else depth
        depth01 = torch.empty((H, W), device=dev, dtype=torch.float32) if depth01 is None else depth01
        g = gaussians_struct(params)
        c = camera_struct(cam)
        fn = "splash_render_forward_pixel" if pixel else "splash_render_forward"
        rc = getattr(_abi.lib(), fn)(self._ctx, st.handle, ctypes.byref(g), medium.data_ptr(), ctypes.byref(c),
                                     image.data_ptr(), _abi.ptr(depth), _abi.ptr(depth01), _stream())
        _abi.check(rc, fn)
        st.shape = (params["means"].shape[0], H, W)
        return image, depth, depth01

    def render(self, params: dict, medium: torch.Tensor, cam: scenes.Camera):
        st = self.state()
        return self.forward(st, params, medium, cam)

    def render_clean(self, params: dict, cam: scenes.Camera):
        """The scene without water: Eq. 5 with beta_D = beta_B = B_inf = 0,
        i.e. the plain composite of Eq. 1. Returns (image, depth, depth01)."""
        return self.render(params, torch.zeros(9, device="cuda"), cam)

    def restore(self, image: torch.Tensor, depth: torch.Tensor, medium: torch.Tensor, out=None) -> torch.Tensor:
        """Water removed from `image` [3,H,W] given a depth map [H,W] and the
        medium [9]: max(I - B_inf (1 - e^{-beta_B z}), 0) e^{beta_D z}."""
        _check_tensor(image, "image")
        H, W = image.shape[1:]
        _check_tensor(depth, "depth", (H, W))
        _check_tensor(medium, "medium", (9,))
        out = torch.empty_like(image) if out is None else out
        _check_tensor(out, "out", (3, H, W))
        rc = _abi.lib().splash_restore(image.data_ptr(), depth.data_ptr(), medium.data_ptr(), int(W), int(H),
                                       out.data_ptr(), _stream())
        _abi.check(rc, "splash_restore")
        return out

    def backward(self, st: State, params: dict, medium: torch.Tensor, cam: scenes.Camera, dL_dimage,
                 dL_ddepth=None, dL_ddepth01=None, grads: dict | None = None, pixel: bool = False) -> dict:
        H, W = cam.height, cam.width
        _check_tensor(dL_dimage, "dL_dimage", (3, H, W))
        if dL_ddepth is not None:
            _check_tensor(dL_ddepth, "dL_ddepth", (H, W))
        if dL_ddepth01 is not None:
            _check_tensor(dL_ddepth01, "dL_ddepth01", (H, W))
        if grads is None:
            grads = {k: torch.empty_like(params[k]) for k in PARAM_NAMES}
            grads["medium"] = torch.empty_like(medium)
        gs = _abi.Grads(*(grads[k].data_ptr() if grads.get(k) is not None else None
                          for k in PARAM_NAMES + ("medium",)))
        g = gaussians_struct(params)
        c = camera_struct(cam)
        fn = "splash_render_backward_pixel" if pixel else "splash_render_backward"
        rc = getattr(_abi.lib(), fn)(self._ctx, st.handle, ctypes.byref(g), medium.data_ptr(), ctypes.byref(c),
                                     dL_dimage.data_ptr(), _abi.ptr(dL_ddepth), _abi.ptr(dL_ddepth01),
                                     ctypes.byref(gs), _stream())
        _abi.check(rc, fn)
        return grads

    def backward_adam(self, st: State, params: dict, medium: torch.Tensor, cam: scenes.Camera, dL_dimage,
                      m: dict, v: dict, lr: dict, step: int, betas=(0.9, 0.999), eps: float = 1e-15,
                      medium_min: float | None = 0.0, dL_ddepth=None, dL_ddepth01=None, grad_medium=None,
                      prior: torch.Tensor | None = None, lambda_est: float = 0.1,
                      densify_stats: torch.Tensor | None = None, pixel: bool = False):
        """Fused training-step backward: gradients of the last forward on `st`
        followed by one Adam step applied in place to params/medium and the
        moment dicts m, v (keys PARAM_NAMES + 'medium'). With `prior` (device
        float32[6] = beta_B_hat, B_inf_hat, e.g. backscatter.prior_of(result)),
        the L_best term of Eq. 9 weighted by lambda_est joins the medium
        gradient. densify_stats ([n, 2] float32) accumulates the densification
        statistics (see densify_plan)."""
        H, W = cam.height, cam.width
        _check_tensor(dL_dimage, "dL_dimage", (3, H, W))
        names = PARAM_NAMES + ("medium",)
        tens = dict(params)
        tens["medium"] = medium
        for k in names:
            _check_tensor(tens[k], k)
            _check_tensor(m[k], f"m[{k}]", tuple(tens[k].shape))
            _check_tensor(v[k], f"v[{k}]", tuple(tens[k].shape))
        pb = _abi.ParamBuffers(*(tens[k].data_ptr() for k in names))
        cfg = _abi.AdamConfig(_abi.ParamBuffers(*(m[k].data_ptr() for k in names)),
                              _abi.ParamBuffers(*(v[k].data_ptr() for k in names)),
                              float(lr["means"]), float(lr["log_scales"]), float(lr["quats"]),
                              float(lr["opacity_logits"]), float(lr["sh"]), float(lr["medium"]),
                              float(betas[0]), float(betas[1]), float(eps), int(step),
                              0 if medium_min is None else 1, float(medium_min or 0.0), _abi.ptr(prior),
                              float(lambda_est), _abi.ptr(densify_stats))
        if densify_stats is not None:
            _check_tensor(densify_stats, "densify_stats", (params["means"].shape[0], 2))
        if prior is not None:
            _check_tensor(prior, "prior", (6,))
        c = camera_struct(cam)
        fn = "splash_render_backward_adam_pixel" if pixel else "splash_render_backward_adam"
        rc = getattr(_abi.lib(), fn)(self._ctx, st.handle, ctypes.byref(pb), params["means"].shape[0],
                                     int(params["sh_degree"]), ctypes.byref(c), dL_dimage.data_ptr(),
                                     _abi.ptr(dL_ddepth), _abi.ptr(dL_ddepth01), ctypes.byref(cfg),
                                     _abi.ptr(grad_medium), _stream())
        _abi.check(rc, fn)

    def state_array(self, st: State, field: str, dtype=torch.int32, shape=None) -> torch.Tensor:
        """Copy of one forward-state buffer (see splash_state_copy)."""
        info = _abi.StateInfo()
        _abi.check(_abi.lib().splash_state_get_info(st.handle, ctypes.byref(info)), "splash_state_get_info")
        n, K = info.n_gaussians, info.n_keys
        tiles = info.tiles_x * info.tiles_y
        _, H, W = st.shape
        sizes = {"tile_ids": (K,), "gauss_ids": (K,), "ranges": (tiles, 2), "depth_keys": (n,), "tiles_touched": (n,),
                 "records": (n, 12), "final_T": (H, W), "acc_alpha": (H, W), "n_last": (H, W), "n_walk": (H, W),
                 "rects": (n, 2)}
        floaty = field in ("records", "final_T", "acc_alpha")
        out = torch.empty(sizes[field], dtype=torch.float32 if floaty else torch.int32, device="cuda")
        rc = _abi.lib().splash_state_copy(st.handle, _abi.FIELDS[field], out.data_ptr(), out.numel() * 4, _stream())
        _abi.check(rc, "splash_state_copy")
        return out if floaty else out.view(dtype)

    def info(self, st: State) -> dict:
        info = _abi.StateInfo()
        _abi.check(_abi.lib().splash_state_get_info(st.handle, ctypes.byref(info)), "splash_state_get_info")
        return {"n_keys": info.n_keys, "tiles_x": info.tiles_x, "tiles_y": info.tiles_y, "tile_w": info.tile_w,
                "tile_h": info.tile_h, "n_gaussians": info.n_gaussians}

    # -- training-step pieces
    def loss(self, st: State, image: torch.Tensor, target: torch.Tensor, lam: float = 0.2, need_grad: bool = True,
             loss_out: torch.Tensor | None = None, grad_out: torch.Tensor | None = None):
        _check_tensor(image, "image")
        _check_tensor(target, "target", tuple(image.shape))
        C, H, W = image.shape
        loss = torch.empty(1, device=image.device, dtype=torch.float32) if loss_out is None else loss_out
        grad = (torch.empty_like(image) if grad_out is None else grad_out) if need_grad else None
        rc = _abi.lib().splash_loss_l1_ssim(self._ctx, st.handle, image.data_ptr(), target.data_ptr(), C, H, W,
                                            float(lam), loss.data_ptr(), _abi.ptr(grad), _stream())
        _abi.check(rc, "splash_loss_l1_ssim")
        return loss, grad

    def sort_pairs(self, st: State, keys: torch.Tensor, vals: torch.Tensor | None = None, bits: int = 32):
        n = keys.numel()
        ko = torch.empty_like(keys)
        vo = torch.empty(n, dtype=torch.int32, device=keys.device)
        rc = _abi.lib().splash_sort_pairs_u32(self._ctx, st.handle, keys.data_ptr(), _abi.ptr(vals), ko.data_ptr(),
                                              vo.data_ptr(), n, int(bits), _stream())
        _abi.check(rc, "splash_sort_pairs_u32")
        return ko, vo

    def profile(self, on: bool = True, stages=None):
        """Stage timing on (clears the totals); `stages` (names from
        _abi.STAGES) restricts it to those stages, None times all."""
        mask = 0xFFFFFFFF if stages is None else sum(1 << _abi.STAGES.index(s) for s in stages)
        _abi.check(_abi.lib().splash_profile_mask(self._ctx, mask), "splash_profile_mask")
        _abi.check(_abi.lib().splash_profile_enable(self._ctx, int(on)), "splash_profile_enable")

    def profile_read(self) -> dict:
        ms = (ctypes.c_double * len(_abi.STAGES))()
        cnt = (ctypes.c_int64 * len(_abi.STAGES))()
        _abi.check(_abi.lib().splash_profile_read(self._ctx, ms, cnt), "splash_profile_read")
        return {s: (ms[i], cnt[i]) for i, s in enumerate(_abi.STAGES)}

    def sync_status(self):
        _abi.check(_abi.lib().splash_sync_status(self._ctx, _stream()), "splash_sync_status")


class Batch:
    """Many views of one scene rendered and differentiated as one unit (one
    persistent blend launch each way, no host synchronisation after
    calibrate(): forward/backward can be captured in a CUDA graph)."""

    def __init__(self, renderer: Renderer, cams: list):
        self.r = renderer
        self.cams = list(cams)
        arr = (_abi.Camera * len(cams))(*[camera_struct(c) for c in cams])
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().splash_batch_create(renderer._ctx, len(cams), arr, ctypes.byref(h)), "splash_batch_create")
        self._h = h
        self.images = None

    def close(self):
        if self._h:
            _abi.lib().splash_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def calibrate(self, params: dict, medium: torch.Tensor, headroom: float = 1.25):
        g = gaussians_struct(params)
        _abi.check(_abi.lib().splash_batch_calibrate(self._h, ctypes.byref(g), medium.data_ptr(), float(headroom),
                                                     _stream()), "splash_batch_calibrate")
        dev = medium.device
        self.images = [torch.empty((3, c.height, c.width), device=dev) for c in self.cams]

    def forward(self, params: dict, medium: torch.Tensor, images=None, depths=None, depth01s=None):
        """Renders every view into ``images`` (default: the batch's own
        buffers); ``depths`` / ``depth01s``, lists of [H_v, W_v] device
        tensors (entries may be None), receive the Eq. 6 depth maps."""
        images = images if images is not None else self.images
        V = len(images)
        arr = lambda ts: None if ts is None else (ctypes.c_void_p * V)(*[_abi.ptr(t) for t in ts])
        g = gaussians_struct(params)
        _abi.check(_abi.lib().splash_batch_forward(self._h, ctypes.byref(g), medium.data_ptr(), arr(images),
                                                   arr(depths), arr(depth01s), _stream()), "splash_batch_forward")
        return images

    def backward(self, params: dict, medium: torch.Tensor, dL_dimages: list, grads: dict | None = None) -> dict:
        if grads is None:
            grads = {k: torch.empty_like(params[k]) for k in PARAM_NAMES}
            grads["medium"] = torch.empty_like(medium)
        ptrs = (ctypes.c_void_p * len(dL_dimages))(*[t.data_ptr() for t in dL_dimages])
        gs = _abi.Grads(*(grads[k].data_ptr() if grads.get(k) is not None else None for k in PARAM_NAMES + ("medium",)))
        g = gaussians_struct(params)
        _abi.check(_abi.lib().splash_batch_backward(self._h, ctypes.byref(g), medium.data_ptr(), ptrs, ctypes.byref(gs),
                                                    _stream()), "splash_batch_backward")
        return grads

    def pair_counts(self):
        V = len(self.cams)
        em, cap = (ctypes.c_int64 * V)(), (ctypes.c_int64 * V)()
        _abi.check(_abi.lib().splash_batch_pair_counts(self._h, em, cap, _stream()), "splash_batch_pair_counts")
        return list(em), list(cap)


def kernel_launches() -> int:
    return int(_abi.lib().splash_kernel_launches())


def densify(renderer: "Renderer", params: dict, m: dict, v: dict, stats: torch.Tensor, noise: torch.Tensor,
            extent: float, grad_threshold: float = 0.0002, min_opacity: float = 0.1, percent_dense: float = 0.01):
    """One densification step (prune / clone / split, see splash_densify_plan):
    returns new (params, m, v) dicts for the Gaussian groups (medium and other
    entries of the dicts are carried over unchanged). noise: [n, 2, 3] standard
    normals for the split samples. Synchronises the stream (the new count)."""
    n = params["means"].shape[0]
    _check_tensor(stats, "stats", (n, 2))
    _check_tensor(noise, "noise", (n, 2, 3))
    opt = _abi.DensifyOptions(float(grad_threshold), float(min_opacity), float(percent_dense), float(extent))
    n_new = ctypes.c_int64()
    L = _abi.lib()
    _abi.check(L.splash_densify_plan(renderer._ctx, params["log_scales"].data_ptr(), params["opacity_logits"].data_ptr(),
                                     stats.data_ptr(), n, ctypes.byref(opt), ctypes.byref(n_new), _stream()),
               "splash_densify_plan")
    nn = int(n_new.value)
    deg = int(params["sh_degree"])
    shapes = {"means": (nn, 3), "log_scales": (nn, 3), "quats": (nn, 4), "opacity_logits": (nn,),
              "sh": (nn, (deg + 1) ** 2, 3)}
    new = [{k: torch.empty(sh, device="cuda") for k, sh in shapes.items()} for _ in range(3)]
    buf = lambda d: _abi.ParamBuffers(*(d[k].data_ptr() for k in PARAM_NAMES), None)
    _abi.check(L.splash_densify_apply(renderer._ctx, ctypes.byref(buf(params)), ctypes.byref(buf(m)), ctypes.byref(buf(v)),
                                      n, deg, noise.data_ptr(), ctypes.byref(buf(new[0])), ctypes.byref(buf(new[1])),
                                      ctypes.byref(buf(new[2])), nn, _stream()), "splash_densify_apply")
    for src, dst in zip((params, m, v), new):
        for k, val in src.items():
            if k not in shapes:
                dst[k] = val
    return tuple(new)


def mcmc_relocate(renderer: "Renderer", params: dict, m: dict, v: dict, uniforms: torch.Tensor,
                  min_opacity: float = 0.005) -> int:
    """One MCMC relocation (see splash_mcmc_relocate), in place on the
    parameter and moment dicts; uniforms: [n] floats in [0, 1). Returns the
    number of dead Gaussians relocated (synchronises the stream)."""
    n = params["means"].shape[0]
    _check_tensor(uniforms, "uniforms", (n,))
    buf = lambda d: _abi.ParamBuffers(*(d[k].data_ptr() for k in PARAM_NAMES), None)
    nd = ctypes.c_int64()
    _abi.check(_abi.lib().splash_mcmc_relocate(renderer._ctx, ctypes.byref(buf(params)), ctypes.byref(buf(m)),
                                               ctypes.byref(buf(v)), n, int(params["sh_degree"]), uniforms.data_ptr(),
                                               float(min_opacity), ctypes.byref(nd), _stream()), "splash_mcmc_relocate")
    return int(nd.value)


def mcmc_noise(params: dict, eta: torch.Tensor, lr: float, lambda_noise: float = 5e5):
    """The MCMC position noise (see splash_mcmc_noise), in place on the means;
    eta: [n, 3] standard normals."""
    n = params["means"].shape[0]
    _check_tensor(eta, "eta", (n, 3))
    _abi.check(_abi.lib().splash_mcmc_noise(params["means"].data_ptr(), params["log_scales"].data_ptr(),
                                            params["quats"].data_ptr(), params["opacity_logits"].data_ptr(),
                                            eta.data_ptr(), n, float(lr), float(lambda_noise), _stream()),
               "splash_mcmc_noise")


def opacity_reset(logits: torch.Tensor, m: torch.Tensor | None = None, v: torch.Tensor | None = None,
                  max_opacity: float = 0.01):
    """The schedule's opacity reset: opacities capped at max_opacity, the
    opacity group's Adam moments (if given) set to zero. In place."""
    _check_tensor(logits, "logits")
    for t, name in ((m, "m"), (v, "v")):
        if t is not None:
            _check_tensor(t, name, tuple(logits.shape))
    rc = _abi.lib().splash_opacity_reset(logits.data_ptr(), _abi.ptr(m), _abi.ptr(v), logits.numel(),
                                         float(max_opacity), _stream())
    _abi.check(rc, "splash_opacity_reset")


def adam_step(groups, step: int, betas=(0.9, 0.999), eps: float = 1e-15):
    """groups: list of dicts {param, grad, m, v, lr, clamp_min (optional)}."""
    if len(groups) > _abi.ADAM_MAX_GROUPS:
        raise ValueError("too many Adam groups")
    arr = (_abi.AdamGroup * len(groups))()
    for i, g in enumerate(groups):
        for k in ("param", "grad", "m", "v"):
            _check_tensor(g[k], f"adam {k}")
        cm = g.get("clamp_min")
        arr[i] = _abi.AdamGroup(g["param"].data_ptr(), g["grad"].data_ptr(), g["m"].data_ptr(), g["v"].data_ptr(),
                                g["param"].numel(), float(g["lr"]), float(cm if cm is not None else 0.0),
                                1 if cm is not None else 0)
    rc = _abi.lib().splash_adam_step(arr, len(groups), int(step), float(betas[0]), float(betas[1]), float(eps), _stream())
    _abi.check(rc, "splash_adam_step")


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, cam, sh_degree, means, log_scales, quats, opacity_logits, sh, medium):
        params = {"means": means, "log_scales": log_scales, "quats": quats, "opacity_logits": opacity_logits, "sh": sh,
                  "sh_degree": sh_degree}
        st = renderer.state()
        img, depth, depth01 = renderer.forward(st, params, medium, cam)
        ctx.renderer, ctx.cam, ctx.st, ctx.sh_degree = renderer, cam, st, sh_degree
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh, medium)
        return img, depth, depth01

    @staticmethod
    def backward(ctx, g_img, g_depth, g_depth01):
        means, log_scales, quats, opacity_logits, sh, medium = ctx.saved_tensors
        params = {"means": means, "log_scales": log_scales, "quats": quats, "opacity_logits": opacity_logits, "sh": sh,
                  "sh_degree": ctx.sh_degree}
        dev = medium.device
        g_img = torch.zeros((3, ctx.cam.height, ctx.cam.width), device=dev) if g_img is None else g_img.contiguous()
        g_depth = None if g_depth is None else g_depth.contiguous()
        g_depth01 = None if g_depth01 is None else g_depth01.contiguous()
        grads = ctx.renderer.backward(ctx.st, params, medium, ctx.cam, g_img, g_depth, g_depth01)
        ctx.st = None
        return (None, None, None, grads["means"], grads["log_scales"], grads["quats"], grads["opacity_logits"],
                grads["sh"], grads["medium"])


def render(params: dict, medium: torch.Tensor, cam: scenes.Camera, renderer: Renderer):
    """Differentiable render: returns (image [3,H,W], depth [H,W], depth01 [H,W])."""
    return _RenderFn.apply(renderer, cam, int(params["sh_degree"]), params["means"], params["log_scales"],
                           params["quats"], params["opacity_logits"], params["sh"], medium)
