"""The device planner of Algorithm 2 (Section IV-A's greedy extraction) against the oracle's plan,
element by element: every [start, stop, basecase] triple and the height bound h that the GPU used
(read back through ``arbgpu_last_plans``) must equal ``oracle.alg2.plan`` on the same inputs, and
the results must contain the exact product within the accuracy bound.  With the inner ordering of
Section IV-B on (the default), the order, the inner scaling exponents and the blocks must equal
``oracle.alg2.plan_ordered``; a real product left with one full block over that order is rounded
once from its exact integer product, so its midpoints are RNE_p of the exact sum."""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import alg2
from synth import random_balls
from synth.workloads import complex_matmul_laplace
from tests.test_gpu_block import (band_case, check_bounds, check_complex, check_entries,
                                  jump_case, run_cmm, run_mm)
from tests.gpu_util import env
from tests.test_oracle_alg2 import TALL_PLANS, _greedy_case, _tall_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def structured_real(seed, n, p=128):
    """Exponents c_k + U[-4, 4] with c_k ~ Laplace(40) along the inner index (the structured
    complex workload's recipe for one real product)."""
    rng = np.random.default_rng(seed)
    c = np.clip(np.rint(rng.laplace(0, 40, size=n)), -200, 200).astype(np.int64)
    ea = np.clip(c[None, :] + rng.integers(-4, 4, size=(n, n), endpoint=True), -200, 200)
    cb = np.clip(np.rint(rng.laplace(0, 40, size=n)), -200, 200).astype(np.int64)
    eb = np.clip(cb[:, None] + rng.integers(-4, 4, size=(n, n), endpoint=True), -200, 200)
    A = random_balls(rng, n * n, 2, 128, exps=ea.reshape(-1), rad_bits=120)
    B = random_balls(rng, n * n, 2, 128, exps=eb.reshape(-1), rad_bits=120)
    return A, B


def _case(kind):
    if kind in TALL_PLANS:
        return _tall_case(kind)
    if kind == "jump":
        A, B = jump_case(4, 24, 100, 20, [35], 64, rad=60)
        return A, B, 24, 100, 20, 64
    if kind == "band":
        A, B = band_case(5, 40, 180, 36, 60, 120, nl=2, rad=120)
        return A, B, 40, 180, 36, 128
    if kind == "drift":
        return _greedy_case(True)
    if kind == "iid":
        return _greedy_case(False)
    if kind == "structured":
        A, B = structured_real(7, 160)
        return A, B, 160, 160, 160, 128
    assert kind == "single"
    rng = np.random.default_rng(11)
    A = random_balls(rng, 70 * 100, 2, 128, -20, 20, rad_bits=120)
    B = random_balls(rng, 100 * 90, 2, 128, -20, 20, rad_bits=120)
    return A, B, 70, 100, 90, 128


def _sample(M, N, count, seed):
    if M * N <= count:
        return [(i, j) for i in range(M) for j in range(N)]
    rng = np.random.default_rng(seed)
    return [(int(a), int(b)) for a, b in zip(rng.integers(0, M, count), rng.integers(0, N, count))]


@pytest.fixture
def contiguous():
    """The inner index in its own order, every input bit kept (no negligible-limb omission)."""
    with env(ARBGPU_INNER_ORDER="0", ARBGPU_OMIT="0"):
        yield


@pytest.mark.parametrize("kind", sorted(TALL_PLANS) + ["jump", "band", "drift", "iid",
                                                       "structured", "single"])
def test_device_plan_equals_oracle_plan(arb, contiguous, kind):
    A, B, M, K, N, p = _case(kind)
    h, blocks = alg2.plan(A, B, M, K, N, p)
    out, _ = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK)
    plans = arb.default_context().last_plans()
    assert plans == [dict(kind=0, h=h, K=K, blocks=blocks)]
    if kind in TALL_PLANS:
        assert blocks == TALL_PLANS[kind]
    check_bounds(out, A, B, M, K, N, p, _sample(M, N, 150, 3))
    if blocks == [(0, K, False)]:  # one block: exactly rounded
        check_entries(out, A, B, M, K, N, p, _sample(M, N, 60, 4), (p + 63) // 64)


def test_device_plans_of_a_complex_product(arb, contiguous):
    """The four real products of a complex product (Ar Br, Ai Bi, Ar Bi, Ai Br), each planned on
    its own (the structured complex Laplace workload at N = 128)."""
    case = complex_matmul_laplace(n=128, structured=True)
    n, p = 128, 128
    outs, _ = run_cmm(arb, case.A, case.B, n, n, n, p, arb.ALG_BLOCK)
    plans = arb.default_context().last_plans()
    want = []
    for xa, yb in ((0, 0), (1, 1), (0, 1), (1, 0)):
        h, blocks = alg2.plan(case.A[xa], case.B[yb], n, n, n, p)
        want.append(dict(kind=0, h=h, K=n, blocks=blocks))
    assert plans == want
    assert any(len(w["blocks"]) > 1 for w in want)
    check_complex(outs, case.A, case.B, n, n, n, p, _sample(n, n, 40, 5))


def test_device_plan_of_the_complex_product_by_eq2(arb):
    """With ARBGPU_MM_COMPLEX_3M and one scaling per row and column shared by both parts that fits
    one block, the record is that shared block under the bound of the parts' precisions, which is
    the plan ``plan_complex_shared`` gives."""
    rng = np.random.default_rng(161)
    M, K, N, p = 70, 100, 90, 256
    A2 = [random_balls(rng, M * K, 4, 256, -20, 20, rad_bits=248) for _ in "ri"]
    B2 = [random_balls(rng, K * N, 4, 256, -20, 20, rad_bits=248) for _ in "ri"]
    outs, names = run_cmm(arb, A2, B2, M, K, N, p, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    assert "z3m" in names
    h, blocks = alg2.plan_complex_shared(A2, B2, M, K, N, p)
    assert blocks == [(0, K, False)]
    assert arb.default_context().last_plans() == [dict(kind=2, h=h, K=K, blocks=blocks)]
    check_complex(outs, A2, B2, M, K, N, p, _sample(M, N, 30, 6))


def complex_bands(seed, M, K, N, bands, nl=2, rad=120):
    """Complex operands: the columns lo..hi-1 of A's real part (first range) and of its imaginary
    part (second range) sit 2^900 higher than the rest; B is uniformly scaled."""
    rng = np.random.default_rng(seed)
    A2, B2 = [], []
    for lo, hi in bands:
        ea = rng.integers(-5, 5, size=M * K)
        for k in range(lo, hi):
            ea[np.arange(M) * K + k] += 900
        A2.append(random_balls(rng, M * K, nl, 64 * nl, exps=ea, rad_bits=rad, rad_zero_frac=0.5))
        B2.append(random_balls(rng, K * N, nl, 64 * nl, -5, 5, rad_bits=rad, rad_zero_frac=0.5))
    return A2, B2


EQ2_BANDS = {
    "same": ((60, 120), (60, 120)),  # three full blocks shared by the parts
    "apart": ((35, 36), (70, 71)),   # a merged entry taller than h in each part: basecase ranges
    "overlap": ((40, 90), (60, 110)),  # full blocks, forced single indices, basecase ranges
}


@pytest.mark.parametrize("kind", sorted(EQ2_BANDS))
def test_device_plan_of_eq2_over_several_blocks(arb, contiguous, kind):
    """Eq. 2 over several blocks (Section IV-C's second suggestion): the device plans the inner
    range once on the merged entry heights of both parts and the record equals
    ``plan_complex_shared`` element by element; every full block's Re and Im come from three
    exact products (z3m), and every sampled ball of both parts contains the exact complex
    product within the accuracy bound."""
    M, K, N, p = 40, 180, 36, 128
    A2, B2 = complex_bands(31 + len(kind), M, K, N, EQ2_BANDS[kind])
    outs, names = run_cmm(arb, A2, B2, M, K, N, p, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    h, blocks = alg2.plan_complex_shared(A2, B2, M, K, N, p)
    assert len(blocks) > 1
    assert arb.default_context().last_plans() == [dict(kind=2, h=h, K=K, blocks=blocks)]
    assert ("z3m" in names) == any(not b[2] for b in blocks)
    if any(b[2] for b in blocks):
        assert "dot_tile" in names or "dot_fused" in names
    check_complex(outs, A2, B2, M, K, N, p, _sample(M, N, 60, 9))


# ------------------------------------------------------------------ inner ordering (Section IV-B)

@pytest.fixture
def ordered():
    """The inner ordering on, every input bit kept (no negligible-limb omission)."""
    with env(ARBGPU_INNER_ORDER="1", ARBGPU_OMIT="0"):
        yield


def _expected_ordered(A, B, M, K, N, p):
    """The record the GPU must write with the inner ordering on: a product that fits one block
    in its own order keeps that block (kind 0); any other runs over ``plan_ordered`` (kind 1)."""
    h, blocks = alg2.plan(A, B, M, K, N, p)
    if blocks == [(0, K, False)]:
        return dict(kind=0, h=h, K=K, blocks=blocks)
    h, order, g, blocks = alg2.plan_ordered(A, B, M, K, N, p)
    return dict(kind=1, h=h, K=K, blocks=blocks, order=order, g=g)


@pytest.mark.parametrize("kind", ["structured", "band", "jump", "iid", "all_tall"])
def test_inner_ordered_plan_equals_oracle(arb, ordered, kind):
    """Products that need several blocks run over the inner order: the order, the scaling
    exponents g_k and the greedy blocks over that order equal ``plan_ordered``, and every checked
    ball contains the exact product within the accuracy bound."""
    A, B, M, K, N, p = _case(kind)
    want = _expected_ordered(A, B, M, K, N, p)
    assert want["kind"] == 1
    blocks = want["blocks"]
    out, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "gather_inner" in names
    assert arb.default_context().last_plans() == [want]
    check_bounds(out, A, B, M, K, N, p, _sample(M, N, 150, 7))
    if blocks == [(0, K, False)]:
        # one full block over the inner order: rounded once from the exact product
        assert "block_round" in names and "accumulate" not in names
        check_entries(out, A, B, M, K, N, p, _sample(M, N, 80, 8), (p + 63) // 64)
    if kind == "structured":  # ordering leaves almost nothing to the basecase
        base = sum(stop - start for start, stop, b in blocks if b)
        assert base <= K // 10


def test_inner_ordering_is_the_default(arb):
    """Without the environment variable the inner ordering runs for products that need several
    blocks (the structured real product: one full block over the order, exactly rounded)."""
    assert os.environ.get("ARBGPU_INNER_ORDER") is None
    with env(ARBGPU_OMIT="0"):
        _inner_ordering_default(arb)


def _inner_ordering_default(arb):
    A, B, M, K, N, p = _case("structured")
    want = _expected_ordered(A, B, M, K, N, p)
    out, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert arb.default_context().last_plans() == [want]
    assert want["blocks"] == [(0, K, False)]
    check_entries(out, A, B, M, K, N, p, _sample(M, N, 80, 9), (p + 63) // 64)


def test_inner_ordered_complex_product(arb, ordered):
    """The structured complex workload at N = 128 with the inner ordering: each real product's
    record equals ``plan_ordered`` and the balls contain the exact product."""
    case = complex_matmul_laplace(n=128, structured=True)
    n, p = 128, 128
    outs, _ = run_cmm(arb, case.A, case.B, n, n, n, p, arb.ALG_BLOCK)
    plans = arb.default_context().last_plans()
    assert len(plans) == 4
    for rec, (xa, yb) in zip(plans, ((0, 0), (1, 1), (0, 1), (1, 0))):
        assert rec == _expected_ordered(case.A[xa], case.B[yb], n, n, n, p)
    check_complex(outs, case.A, case.B, n, n, n, p, _sample(n, n, 40, 8))


@pytest.mark.parametrize("kind", ["structured", "overlap"])
def test_inner_ordered_eq2_plan_equals_oracle(arb, ordered, kind):
    """Both suggestions together: eq. 2 over blocks planned for both parts at once, over an inner
    order and scaling shared by the parts.  The record (kind 4) equals ``plan_complex_ordered``:
    blocks, order and scaling exponents; the sampled balls contain the exact product within the
    accuracy bound."""
    if kind == "structured":
        case = complex_matmul_laplace(n=128, structured=True)
        A2, B2, M, K, N, p = case.A, case.B, 128, 128, 128, 128
    else:
        M, K, N, p = 40, 180, 36, 128
        A2, B2 = complex_bands(38, M, K, N, EQ2_BANDS[kind])
    outs, names = run_cmm(arb, A2, B2, M, K, N, p, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    h, order, g, blocks = alg2.plan_complex_ordered(A2, B2, M, K, N, p)
    assert arb.default_context().last_plans() == [
        dict(kind=4, h=h, K=K, blocks=blocks, order=order, g=g)]
    assert any(not b[2] for b in blocks) and "z3m" in names
    check_complex(outs, A2, B2, M, K, N, p, _sample(M, N, 60, 10))
