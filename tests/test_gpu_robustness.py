"""Repeatability and the synchronous error paths of the C ABI on the GPU.

Races would show up as run-to-run differences. The integer paths are deterministic by
construction: exact integer sums, and reductions in a fixed order. So two calls on the same inputs
must agree bit for bit in every output field, on each path: one block, several blocks with
basecase dots, classical dots, and the complex product by eq. 2. Argument errors (a workspace
smaller than the query gave, unknown flag bits) return at once, launch nothing and leave the device
status word clear."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from synth import random_balls
from tests.gpu_util import to_raw

pytestmark = pytest.mark.gpu

FIELDS = ("limbs", "exp", "flags", "rad_man", "rad_exp")


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


@pytest.fixture(autouse=True)
def clear_status(arb):
    arb.default_context().status()  # start from a clear status word (it is read and cleared)


def _inputs(arb, seed, M, K, N, p, parts, lo, hi):
    rng = np.random.default_rng(seed)
    nl = (p + 63) // 64
    A = [arb.Balls.from_raw(random_balls(rng, M * K, nl, p, lo, hi, rad_bits=p - 8,
                                         rad_zero_frac=0.5)) for _ in range(parts)]
    B = [arb.Balls.from_raw(random_balls(rng, K * N, nl, p, lo, hi, rad_bits=p - 8,
                                         rad_zero_frac=0.5)) for _ in range(parts)]
    return A, B


@pytest.mark.parametrize("kind", ["block", "several", "dot", "complex3m", "complex3m_several"])
def test_repeated_calls_are_bitwise_identical(arb, kind):
    if kind == "block":
        M, K, N, p, parts, lo, hi, alg, flags = 96, 96, 96, 128, 1, -10, 10, arb.ALG_BLOCK, 0
    elif kind == "several":  # exponents far wider than h: several blocks and basecase dots
        M, K, N, p, parts, lo, hi, alg, flags = 48, 120, 40, 64, 1, -400, 400, arb.ALG_BLOCK, 0
    elif kind == "dot":
        M, K, N, p, parts, lo, hi, alg, flags = 40, 40, 40, 192, 1, -30, 30, arb.ALG_DOT, 0
    elif kind == "complex3m":
        M, K, N, p, parts, lo, hi, alg, flags = (64, 64, 64, 128, 2, -10, 10, arb.ALG_BLOCK,
                                                 arb.MM_COMPLEX_3M)
    else:  # eq. 2 over several blocks shared by the parts
        M, K, N, p, parts, lo, hi, alg, flags = (48, 120, 40, 64, 2, -400, 400, arb.ALG_BLOCK,
                                                 arb.MM_COMPLEX_3M)
    A, B = _inputs(arb, 90, M, K, N, p, parts, lo, hi)
    nl = (p + 63) // 64
    pick = (lambda v: v) if parts == 2 else (lambda v: v[0])
    runs = []
    for _ in range(2):
        C = [arb.Balls.empty(M * N, nl) for _ in range(parts)]
        arb.mat_mul(pick(C), pick(A), pick(B), M, K, N, p, alg=alg, flags=flags)
        runs.append([to_raw(c) for c in C])
    assert arb.default_context().status() == 0
    for a, b in zip(*runs):
        for f in FIELDS:
            assert np.array_equal(getattr(a, f), getattr(b, f)), (kind, f)


def test_short_workspace_is_rejected(arb):
    M = K = N = 64
    p = 128
    A, B = _inputs(arb, 91, M, K, N, p, 1, -10, 10)
    need = arb.mat_mul_workspace_size(M, K, N, p, 2, 2, False, arb.ALG_BLOCK)
    assert need > 0
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    C = arb.Balls.empty(M * N, 2)
    with pytest.raises(arb.ArbgpuError) as e:
        arb.mat_mul(C, A[0], B[0], M, K, N, p, alg=arb.ALG_BLOCK, workspace=ws)
    assert e.value.code == 3  # ARBGPU_ERR_WORKSPACE
    assert arb.default_context().status() == 0


def test_3m_flag_needs_the_workspace_queried_with_it(arb):
    M = K = N = 64
    p = 128
    A, B = _inputs(arb, 92, M, K, N, p, 2, -10, 10)
    need4 = arb.mat_mul_workspace_size(M, K, N, p, 2, 2, True, arb.ALG_BLOCK, 0)
    need3 = arb.mat_mul_workspace_size(M, K, N, p, 2, 2, True, arb.ALG_BLOCK, arb.MM_COMPLEX_3M)
    assert need3 > need4  # the three products' planes
    ws = torch.empty(need4, dtype=torch.uint8, device="cuda")
    C = [arb.Balls.empty(M * N, 2), arb.Balls.empty(M * N, 2)]
    with pytest.raises(arb.ArbgpuError) as e:
        arb.mat_mul(C, A, B, M, K, N, p, alg=arb.ALG_BLOCK, flags=arb.MM_COMPLEX_3M, workspace=ws)
    assert e.value.code == 3  # ARBGPU_ERR_WORKSPACE
    assert arb.default_context().status() == 0


def test_unknown_flag_bits_are_rejected(arb):
    M = K = N = 64
    p = 128
    A, B = _inputs(arb, 93, M, K, N, p, 1, -10, 10)
    C = arb.Balls.empty(M * N, 2)
    with pytest.raises(arb.ArbgpuError) as e:
        arb.mat_mul(C, A[0], B[0], M, K, N, p, alg=arb.ALG_BLOCK, flags=2)
    assert e.value.code == 1  # ARBGPU_ERR_INVALID
    need = arb.mat_mul_workspace_size(M, K, N, p, 2, 2, False, arb.ALG_BLOCK)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(arb.ArbgpuError) as e:  # the same through the product call itself
        arb.mat_mul(C, A[0], B[0], M, K, N, p, alg=arb.ALG_BLOCK, flags=2, workspace=ws)
    assert e.value.code == 1
    assert arb.default_context().status() == 0


def test_reserve_uploads_tables_and_products_still_match(arb):
    """arbgpu_reserve on a fresh context, then the same product there and on the default context:
    bit-identical outputs.  Bad arguments are rejected synchronously."""
    from paper_1901_04289_gb300 import _lib
    ctx = arb.Context()
    try:
        ctx.reserve(256, 512)
        with pytest.raises(_lib.ArbgpuError):
            ctx.reserve(1, 512)
        with pytest.raises(_lib.ArbgpuError):
            ctx.reserve(256, 0)
        A, B = _inputs(arb, 91, 96, 120, 80, 256, 1, -20, 20)
        outs = []
        for c in (ctx, arb.default_context()):
            C = arb.Balls.empty(96 * 80, 4)
            arb.mat_mul(C, A[0], B[0], 96, 120, 80, 256, alg=arb.ALG_BLOCK, ctx=c)
            assert c.status() == 0
            outs.append(to_raw(C))
        for f in FIELDS:
            assert np.array_equal(getattr(outs[0], f), getattr(outs[1], f)), f
    finally:
        ctx.close()
