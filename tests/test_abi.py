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


def test_binding_structs_match_the_compilers_layout():
    """Every ctypes mirror against sizeof / offsetof as the library's own
    compiler laid the header's structs out (splash_abi_layout), field by
    field, for all thirteen structs."""
    L = _abi.lib()
    ns, no = ctypes.c_int32(), ctypes.c_int32()
    assert L.splash_abi_layout(None, None, None, ctypes.byref(ns), ctypes.byref(no)) == _abi.OK
    assert ns.value == len(_abi.LAYOUT_ORDER) == 13
    sizes, nf = (ctypes.c_int32 * ns.value)(), (ctypes.c_int32 * ns.value)()
    offs = (ctypes.c_int32 * no.value)()
    assert L.splash_abi_layout(sizes, nf, offs, ctypes.byref(ns), ctypes.byref(no)) == _abi.OK
    k = 0
    for i, T in enumerate(_abi.LAYOUT_ORDER):
        assert ctypes.sizeof(T) == sizes[i], (T.__name__, ctypes.sizeof(T), sizes[i])
        fields = [name for name, _ in T._fields_]
        assert len(fields) == nf[i], (T.__name__, fields, nf[i])
        for name in fields:
            assert getattr(T, name).offset == offs[k], (T.__name__, name, getattr(T, name).offset, offs[k])
            k += 1
    assert k == no.value


def test_library_reports_missing_gpu_as_an_error_not_a_fallback():
    import torch
    if torch.cuda.is_available():
        return
    L = _abi.lib()
    h = ctypes.c_void_p()
    rc = L.splash_create(None, ctypes.byref(h))
    assert rc == _abi.ERR_CUDA and not h.value
    assert len(L.splash_last_error()) > 0
