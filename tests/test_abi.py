"""The C ABI library builds for sm_103a, loads on a machine without a GPU,
and exports every entry point include/splash.h declares (no compute calls)."""
import ctypes
import os

from paper_2411_19588_b300 import _abi, build


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    syms = _abi.header_symbols()
    assert len(syms) >= 13
    for s in syms:
        assert hasattr(L, s), s
    # the binding declares a signature for every entry point except the message getter
    assert set(syms) - {"splash_last_error", "splash_kernel_launches"} == set(_abi._SIGS)


def test_binding_struct_sizes_match_header_layout():
    # int32 x2 + float x4 + float[12] + float x2
    assert ctypes.sizeof(_abi.Camera) == 4 * (2 + 4 + 12 + 2)
    assert ctypes.sizeof(_abi.Gaussians) == 8 * 5 + 8 + 8
    assert ctypes.sizeof(_abi.Options) == 20
    assert ctypes.sizeof(_abi.AdamGroup) == 8 * 4 + 8 + 4 + 4 + 4 + 4


def test_library_reports_missing_gpu_as_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        return
    L = _abi.lib()
    h = ctypes.c_void_p()
    rc = L.splash_create(None, ctypes.byref(h))
    assert rc == _abi.ERR_CUDA and not h.value
    assert len(L.splash_last_error()) > 0
