"""The allocation-free integer product (arbgpu_int_mat_mul_noalloc), called through the C ABI, must
give exactly what arbgpu_int_mat_mul gives, on two calls in a row.  It is meant for callers that
cannot allocate device memory (their device memory belongs to another allocator's pool, or they
must not enter the CUDA allocator); this file is collected last so that a stop-at-first-failure
run has already run every other test."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCRATCH = 32 << 20  # ARBGPU_NOALLOC_SCRATCH_BYTES


def limb_planes(rng, nl, count):
    return rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, size=(nl, count),
                        dtype=np.int64, endpoint=True)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _call(L, T, tl, X, xl, Y, yl, M, K, N, status):
    import torch
    return L.arbgpu_int_mat_mul_noalloc(_ptr(T), tl, _ptr(X), xl, _ptr(Y), yl, M, K, N,
                                        _ptr(status),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _reference(rng, M, K, N, xl, yl, tl):
    import torch

    import paper_1901_04289_gb300 as arb
    X = torch.from_numpy(limb_planes(rng, xl, M * K)).cuda()
    Y = torch.from_numpy(limb_planes(rng, yl, K * N)).cuda()
    T_ref = torch.zeros((tl, M * N), dtype=torch.int64, device="cuda")
    arb.int_mat_mul(T_ref, tl, X, xl, Y, yl, M, K, N)
    return X, Y, T_ref


def test_noalloc_matches_int_mat_mul_on_two_calls():
    import torch

    import paper_1901_04289_gb300 as arb
    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    rng = np.random.default_rng(20240611)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for M, K, N, xl, yl in [(150, 300, 140, 2, 2), (64, 64, 300, 1, 3)]:
        tl = xl + yl + 1
        X, Y, T_ref = _reference(rng, M, K, N, xl, yl, tl)
        T_new = torch.full((tl, M * N), 7, dtype=torch.int64, device="cuda")
        assert _call(L, T_new, tl, X, xl, Y, yl, M, K, N, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert arb.default_context().status() == 0
        # integer results: the tolerance is zero
        assert torch.equal(T_new, T_ref)


def test_noalloc_without_status_word_and_near_the_scratch_limit():
    """status = NULL on a real product, and a size whose scratch is just under the array."""
    import torch

    import paper_1901_04289_gb300 as arb
    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    rng = np.random.default_rng(77)
    # 1024 x 1024 x 448 with one-limb operands: the digit planes, the digit bytes of the product
    # and the carries come to just under 32 MiB
    M, K, N, xl, yl = 448, 1024, 448, 1, 1
    tl = 3
    need = C.c_size_t(0)
    assert L.arbgpu_int_mat_mul_workspace_size(arb.default_context().handle, xl, yl, M, K, N,
                                               C.byref(need)) == 0
    assert SCRATCH * 3 // 4 < need.value <= SCRATCH
    X, Y, T_ref = _reference(rng, M, K, N, xl, yl, tl)
    for _ in range(2):
        T_new = torch.full((tl, M * N), -3, dtype=torch.int64, device="cuda")
        assert _call(L, T_new, tl, X, xl, Y, yl, M, K, N, None) == 0
        torch.cuda.synchronize()
        assert torch.equal(T_new, T_ref)
    assert arb.default_context().status() == 0


def test_noalloc_empty_and_zero_inner_dimension():
    import torch

    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    rng = np.random.default_rng(5)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    X = torch.from_numpy(limb_planes(rng, 1, 16)).cuda()
    # M = 0 and N = 0: nothing to write
    assert _call(L, None, 2, X, 1, X, 1, 0, 4, 4, status) == 0
    assert _call(L, None, 2, X, 1, X, 1, 4, 4, 0, None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # K = 0: the product is the zero matrix
    T = torch.full((2, 12), 9, dtype=torch.int64, device="cuda")
    assert _call(L, T, 2, None, 1, None, 1, 3, 0, 4, status) == 0
    torch.cuda.synchronize()
    assert int(T.abs().sum().item()) == 0


def test_noalloc_rejects_bad_arguments_and_sizes_beyond_its_scratch():
    import torch

    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    torch.cuda.init()
    assert _call(L, None, 5, None, 2, None, 2, 4096, 4096, 4096, None) == _lib.ERR_LIMIT
    # sizes whose layout would wrap a 64-bit byte count are rejected before it is computed
    assert _call(L, None, 5, None, 32, None, 32, 1 << 30, 1 << 30, 1 << 30, None) == _lib.ERR_LIMIT
    # an output wider than the engine's 68 limbs
    assert _call(L, None, 69, None, 1, None, 1, 4, 4, 4, None) == _lib.ERR_INVALID
