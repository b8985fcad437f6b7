"""ctypes binding of libsplash.so (include/splash.h): struct layouts and
argument marshalling only; every step of the render runs in the library's
CUDA kernels. Loading fails loudly when the library cannot be built or
loaded; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

_lib = None

c_float_p = ctypes.POINTER(ctypes.c_float)
c_u32_p = ctypes.POINTER(ctypes.c_uint32)

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_CAPACITY, ERR_TIMEOUT, ERR_STATE = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "CAPACITY", 5: "TIMEOUT", 6: "STATE"}


class SplashError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12),
                ("z_near", ctypes.c_float), ("z_far", ctypes.c_float)]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("sh_degree", ctypes.c_int32)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("medium", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("spin_limit", ctypes.c_int32),
                ("test_stall_partition", ctypes.c_int32), ("gaussian_batch", ctypes.c_int32)]


class StateInfo(ctypes.Structure):
    _fields_ = [("n_keys", ctypes.c_int64), ("tiles_x", ctypes.c_int32), ("tiles_y", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("n_gaussians", ctypes.c_int64),
                ("tile_ids", ctypes.c_void_p), ("gauss_ids", ctypes.c_void_p), ("ranges", ctypes.c_void_p),
                ("depth_keys", ctypes.c_void_p), ("tiles_touched", ctypes.c_void_p), ("records", ctypes.c_void_p),
                ("final_T", ctypes.c_void_p), ("acc_alpha", ctypes.c_void_p), ("n_last", ctypes.c_void_p),
                ("n_walk", ctypes.c_void_p)]


class AdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("m", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("lr", ctypes.c_float), ("clamp_min", ctypes.c_float),
                ("has_clamp", ctypes.c_int32)]


class ParamBuffers(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("medium", ctypes.c_void_p)]


class AdamConfig(ctypes.Structure):
    _fields_ = [("m", ParamBuffers), ("v", ParamBuffers), ("lr_means", ctypes.c_float),
                ("lr_log_scales", ctypes.c_float), ("lr_quats", ctypes.c_float), ("lr_opacity_logits", ctypes.c_float),
                ("lr_sh", ctypes.c_float), ("lr_medium", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("step", ctypes.c_int32),
                ("clamp_medium", ctypes.c_int32), ("medium_min", ctypes.c_float), ("prior", ctypes.c_void_p),
                ("lambda_est", ctypes.c_float), ("densify_stats", ctypes.c_void_p)]


class DensifyOptions(ctypes.Structure):
    _fields_ = [("grad_threshold", ctypes.c_float), ("min_opacity", ctypes.c_float), ("percent_dense", ctypes.c_float),
                ("extent", ctypes.c_float)]


BS_MAX_POINTS = 64


class BackscatterOptions(ctypes.Structure):
    _fields_ = [("resized_height", ctypes.c_int32), ("edges", ctypes.c_int32), ("intervals", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("p_dark", ctypes.c_double), ("b_max", ctypes.c_float),
                ("beta_max", ctypes.c_float)]


class BackscatterResult(ctypes.Structure):
    _fields_ = [("beta_b", ctypes.c_float * 3), ("b_inf", ctypes.c_float * 3), ("residual", ctypes.c_float * 3),
                ("n_points", ctypes.c_int32 * 3), ("n_dark", ctypes.c_int32), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("point_z", (ctypes.c_float * BS_MAX_POINTS) * 3), ("point_v", (ctypes.c_float * BS_MAX_POINTS) * 3)]


ADAM_MAX_GROUPS = 8


class MlpParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


class MlpAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


MLP_IN, MLP_ROW, MLP_HIDDEN, MLP_OUT = 3080, 3136, 128, 9

# the mirrors of the header's structs, in the order splash_abi_layout reports them
LAYOUT_ORDER = (Camera, Gaussians, Grads, Options, ParamBuffers, AdamConfig, StateInfo, AdamGroup, MlpParams, MlpAdam,
                DensifyOptions, BackscatterOptions, BackscatterResult)

_SIGS = {
    "splash_mcmc_relocate": [ctypes.c_void_p, ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers),
                             ctypes.POINTER(ParamBuffers), ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.c_float, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p],
    "splash_mcmc_noise": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_void_p],
    "splash_abi_layout": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int32)],
    "splash_create": [ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)],
    "splash_destroy": [ctypes.c_void_p],
    "splash_state_create": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)],
    "splash_state_destroy": [ctypes.c_void_p],
    "splash_render_forward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p,
                              ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "splash_render_backward": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p,
                               ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(Grads), ctypes.c_void_p],
    "splash_render_forward_pixel": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p,
                                    ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p],
    "splash_render_backward_pixel": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p,
                                     ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.POINTER(Grads), ctypes.c_void_p],
    "splash_render_backward_adam_pixel": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ParamBuffers),
                                          ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Camera), ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(AdamConfig),
                                          ctypes.c_void_p, ctypes.c_void_p],
    "splash_state_get_info": [ctypes.c_void_p, ctypes.POINTER(StateInfo)],
    "splash_render_backward_adam": [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ParamBuffers), ctypes.c_int64,
                                    ctypes.c_int32, ctypes.POINTER(Camera), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.POINTER(AdamConfig), ctypes.c_void_p, ctypes.c_void_p],
    "splash_loss_l1_ssim": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                            ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p],
    "splash_adam_step": [ctypes.POINTER(AdamGroup), ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                         ctypes.c_float, ctypes.c_void_p],
    "splash_sort_pairs_u32": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p],
    "splash_sync_status": [ctypes.c_void_p, ctypes.c_void_p],
    "splash_state_copy": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p],
    "splash_profile_enable": [ctypes.c_void_p, ctypes.c_int32],
    "splash_profile_read": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
    "splash_profile_mask": [ctypes.c_void_p, ctypes.c_uint32],
    "splash_batch_create": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(Camera), ctypes.POINTER(ctypes.c_void_p)],
    "splash_batch_destroy": [ctypes.c_void_p],
    "splash_batch_calibrate": [ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p, ctypes.c_float,
                               ctypes.c_void_p],
    "splash_batch_forward": [ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "splash_batch_backward": [ctypes.c_void_p, ctypes.POINTER(Gaussians), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(Grads), ctypes.c_void_p],
    "splash_batch_pair_counts": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.c_void_p],
    "splash_featurise": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                         ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p],
    "splash_gemm_bf16": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                         ctypes.c_void_p],
    "splash_mlp_create": [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)],
    "splash_mlp_destroy": [ctypes.c_void_p],
    "splash_mlp_set_params": [ctypes.c_void_p, ctypes.POINTER(MlpParams), ctypes.c_void_p],
    "splash_mlp_get_params": [ctypes.c_void_p, ctypes.POINTER(MlpParams), ctypes.c_void_p],
    "splash_mlp_predict": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
    "splash_mlp_step": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                        ctypes.POINTER(MlpAdam), ctypes.c_void_p, ctypes.POINTER(MlpParams), ctypes.c_void_p],
    "splash_backscatter_estimate": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(BackscatterOptions), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p],
    "splash_backscatter_prior": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p],
    "splash_densify_plan": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                            ctypes.POINTER(DensifyOptions), ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p],
    "splash_densify_apply": [ctypes.c_void_p, ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers),
                             ctypes.POINTER(ParamBuffers), ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers), ctypes.POINTER(ParamBuffers),
                             ctypes.c_int64, ctypes.c_void_p],
    "splash_opacity_reset": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_float,
                             ctypes.c_void_p],
    "splash_restore": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                       ctypes.c_void_p, ctypes.c_void_p],
    "splash_sort_pairs_u32_noalloc": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p],
}

NOALLOC_MAX_PAIRS = 1 << 20

STAGES = ["preprocess", "depth_sort", "scan", "emit", "tile_sort", "ranges", "blend_fwd", "blend_bwd",
          "preprocess_bwd", "medium_reduce", "loss", "backscatter",
          "bs_resize"]

FIELDS = {"tile_ids": 0, "gauss_ids": 1, "ranges": 2, "depth_keys": 3, "tiles_touched": 4, "records": 5,
          "final_T": 6, "acc_alpha": 7, "n_last": 8, "n_walk": 9, "rects": 10}


def header_symbols() -> list[str]:
    """Function names declared in include/splash.h."""
    with open(os.path.join(_build.INCLUDE, "splash.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:splash_status|const char \*|uint64_t)\s*(splash_\w+)\s*\(", text, re.M)))


def lib():
    """Build (if stale) and load libsplash.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.splash_last_error.argtypes = []
        L.splash_last_error.restype = ctypes.c_char_p
        L.splash_kernel_launches.argtypes = []
        L.splash_kernel_launches.restype = ctypes.c_uint64
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != OK:
        msg = lib().splash_last_error().decode(errors="replace")
        raise SplashError(status, where, msg)


def ptr(t) -> int | None:
    """Device address of a tensor (None for None)."""
    if t is None:
        return None
    return t.data_ptr()
