"""splash_sort_pairs_u32_noalloc: the pair sort for callers that cannot
allocate device memory (its scratch is a static device array). Called
through the C ABI and compared bit for bit with the allocating entry point,
splash_sort_pairs_u32, on two calls in a row, and with numpy's stable
argsort of the masked keys. This file is collected last so that a failure
here leaves every other test already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_19588_b300 import _abi
from paper_2411_19588_b300 import render as R

pytestmark = pytest.mark.gpu


def _noalloc(L, keys, vals, bits):
    n = keys.numel()
    ko = torch.empty_like(keys)
    vo = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    rc = L.splash_sort_pairs_u32_noalloc(keys.data_ptr(), None if vals is None else vals.data_ptr(), ko.data_ptr(),
                                         vo.data_ptr(), n, bits, status.data_ptr(),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _abi.check(rc, "splash_sort_pairs_u32_noalloc")
    return ko, vo, status


def _numpy_reference(keys, vals, bits):
    k = keys.cpu().numpy().view(np.uint32)
    masked = k & np.uint32((1 << bits) - 1) if bits < 32 else k
    order = np.argsort(masked, kind="stable")
    v = np.arange(k.size, dtype=np.uint32) if vals is None else vals.cpu().numpy().view(np.uint32)
    return k[order], v[order]


def test_noalloc_sort_matches_allocating_sort_twice(cuda_lib):
    L = _abi.lib()
    r = R.Renderer()
    st = r.state()
    rng = np.random.default_rng(2024)
    cases = [(300_001, 20, 1 << 20, True), (_abi.NOALLOC_MAX_PAIRS, 32, 1 << 31, False)]
    for n, bits, distinct, with_vals in cases:  # two calls in a row share the static scratch
        keys = torch.from_numpy(rng.integers(0, distinct, n, dtype=np.int64).astype(np.uint32).view(np.int32)).cuda()
        vals = torch.from_numpy(rng.integers(0, 1 << 31, n, dtype=np.int64).astype(np.int32)).cuda() if with_vals else None
        ko, vo, status = _noalloc(L, keys, vals, bits)
        ref_k, ref_v = r.sort_pairs(st, keys, vals, bits)
        r.sync_status()
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(ko, ref_k) and torch.equal(vo, ref_v)
        np_k, np_v = _numpy_reference(keys, vals, bits)
        np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), np_k)
        np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), np_v)


@pytest.mark.parametrize("n,bits", [(0, 32), (5_000, 0), (1, 7), (4_097, 9)])
def test_noalloc_sort_edge_cases(cuda_lib, n, bits):
    """No pairs; no key bits (the input order is kept and the values are the
    positions); one pair; a ragged partition with a narrow digit."""
    L = _abi.lib()
    rng = np.random.default_rng(n + bits)
    keys = torch.from_numpy(rng.integers(0, 1 << 32, n, dtype=np.int64).astype(np.uint32).view(np.int32)).cuda()
    ko, vo, status = _noalloc(L, keys, None, bits)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    np_k, np_v = _numpy_reference(keys, None, bits)
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), np_k)
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), np_v)


def test_noalloc_sort_rejects_sizes_beyond_its_scratch(cuda_lib):
    L = _abi.lib()
    n = _abi.NOALLOC_MAX_PAIRS + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    rc = L.splash_sort_pairs_u32_noalloc(keys.data_ptr(), None, out.data_ptr(), out.data_ptr(), n, 32, None,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == _abi.ERR_INVALID_ARG
    assert b"static scratch" in L.splash_last_error()
