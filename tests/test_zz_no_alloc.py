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


def limb_planes(rng, nl, count):
    return rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, size=(nl, count),
                        dtype=np.int64, endpoint=True)


def test_noalloc_matches_int_mat_mul_on_two_calls():
    import torch

    import paper_1901_04289_gb300 as arb
    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    rng = np.random.default_rng(20240611)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for M, K, N, xl, yl in [(150, 300, 140, 2, 2), (64, 64, 300, 1, 3)]:
        tl = xl + yl + 1
        X = torch.from_numpy(limb_planes(rng, xl, M * K)).cuda()
        Y = torch.from_numpy(limb_planes(rng, yl, K * N)).cuda()
        T_ref = torch.zeros((tl, M * N), dtype=torch.int64, device="cuda")
        arb.int_mat_mul(T_ref, tl, X, xl, Y, yl, M, K, N)
        T_new = torch.full((tl, M * N), 7, dtype=torch.int64, device="cuda")
        rc = L.arbgpu_int_mat_mul_noalloc(
            C.c_void_p(T_new.data_ptr()), tl, C.c_void_p(X.data_ptr()), xl,
            C.c_void_p(Y.data_ptr()), yl, M, K, N, C.c_void_p(status.data_ptr()),
            C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert arb.default_context().status() == 0
        # integer results: the tolerance is zero
        assert torch.equal(T_new, T_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_1901_04289_gb300 import _lib

    L = _lib.lib()
    torch.cuda.init()
    rc = L.arbgpu_int_mat_mul_noalloc(None, 5, None, 2, None, 2, 4096, 4096, 4096, None, None)
    assert rc == _lib.ERR_LIMIT
