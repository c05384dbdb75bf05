"""The block algorithm (Algorithm 2) on the GPU against the exact oracle: midpoints equal the exactly
rounded value RNE_p(sum_k a_ik b_kj) bit for bit, every ball contains the exact product, and exact
inputs give exact results with zero radius."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import alg1, alg2
from oracle import exact as X
from synth import SEED_BASE, random_balls
from synth.workloads import block_matmul_n512, matmul_uniform
from tests.gpu_util import to_raw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def run_mm(arb, A, B, M, K, N, prec, alg, nl_out=None, trace=False):
    nl_out = nl_out or (prec + 63) // 64
    ctx = arb.default_context()
    C = arb.Balls.empty(M * N, nl_out)
    if trace:
        ctx.trace(True)
    arb.mat_mul(C, arb.Balls.from_raw(A), arb.Balls.from_raw(B), M, K, N, prec, alg=alg)
    st = ctx.status()
    names = [r[0] for r in ctx.trace_read()] if trace else []
    ctx.trace(False)
    assert st == 0
    return to_raw(C), names


def check_entries(out, A, B, M, K, N, prec, entries, nl_out):
    worst_acc = 0.0
    loose = []
    for i, j in entries:
        terms = X.matmul_entry_terms(A, B, K, N, i, j)
        m_ref, r_ref, S, Sabs, R = X.result_exact(terms, prec, nl_out)
        limbs, e, fl = X.encode_mid(m_ref, nl_out)
        idx = i * N + j
        got = ([int(out.limbs[k, idx]) for k in range(nl_out)], int(out.exp[idx]),
               int(out.flags[idx]))
        assert got == (limbs, e, fl), (i, j)
        m, r = X.mid(out, idx), X.rad(out, idx)
        assert X.contains(m, r, S, R), (i, j)
        worst_acc = max(worst_acc, X.accuracy_ratio(m, S, Sabs, prec))
        tight = X.dy_add(R, X.dy_abs(X.dy_add(m, X.dy_neg(S))))
        if tight[0]:
            loose.append(float(X.dy_to_fraction(r) / X.dy_to_fraction(tight)))
    assert worst_acc <= 1.0  # exact rounding: at most 2^-p |S|
    return loose


@pytest.mark.parametrize("M,K,N,prec,spread,rad", [(70, 100, 90, 128, 20, 120),
                                                   (129, 64, 131, 64, 5, 60),
                                                   (40, 257, 33, 256, 30, 250),
                                                   (64, 48, 200, 512, 50, None)])
def test_block_small_exact_rounding(arb, M, K, N, prec, spread, rad):
    rng = np.random.default_rng(M + K + N)
    nl = (prec + 63) // 64
    A = random_balls(rng, M * K, nl, prec, -spread, spread, rad_bits=rad, rad_zero_frac=0.5,
                     zero_frac=0.05)
    B = random_balls(rng, K * N, nl, prec, -spread, spread, rad_bits=rad, rad_zero_frac=0.5,
                     zero_frac=0.05)
    h, blocks = alg2.plan(A, B, M, K, N, prec)
    assert blocks == [(0, K, False)]  # a single exponent block
    out, names = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, trace=True)
    assert any(n.startswith("digit_gemm") for n in names)
    rng2 = np.random.default_rng(1)
    ents = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 150), rng2.integers(0, N, 150))]
    loose = check_entries(out, A, B, M, K, N, prec, ents, nl)
    if loose:
        print("looseness median", np.median(loose), "max", max(loose))
        assert np.median(loose) < 64.0


def test_block_exact_inputs_give_exact_results(arb):
    """64-bit mantissas, narrow exponents, p = 512: the whole exact product fits in p bits, so the
    block result equals the exact value bit for bit and the radius is zero (checks all of T)."""
    rng = np.random.default_rng(3)
    M, K, N, prec = 96, 160, 80, 512
    A = random_balls(rng, M * K, 1, 64, -3, 3)
    B = random_balls(rng, K * N, 1, 64, -3, 3)
    out, _ = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, nl_out=8)
    for i in range(0, M, 7):
        for j in range(0, N, 5):
            S, _, _ = X.dot_terms_exact(X.matmul_entry_terms(A, B, K, N, i, j))
            idx = i * N + j
            assert X.dy_cmp(X.mid(out, idx), S) == 0
            assert int(out.rad_man[idx]) == 0


def test_block_n512_p256_sampled(arb):
    case = block_matmul_n512(prec=256)
    out, names = run_mm(arb, case.A[0], case.B[0], 512, 512, 512, 256, arb.ALG_AUTO, trace=True)
    assert "digit_gemm_mid" in names
    rng = np.random.default_rng(5)
    ents = [(int(a), int(b)) for a, b in zip(rng.integers(0, 512, 120), rng.integers(0, 512, 120))]
    loose = check_entries(out, case.A[0], case.B[0], 512, 512, 512, 256, ents, 4)
    print("looseness median", np.median(loose), "max", max(loose))
    assert np.median(loose) < 64.0


def test_block_n512_p128_sampled(arb):
    case = block_matmul_n512(prec=128)
    out, _ = run_mm(arb, case.A[0], case.B[0], 512, 512, 512, 128, arb.ALG_AUTO)
    rng = np.random.default_rng(6)
    ents = [(int(a), int(b)) for a, b in zip(rng.integers(0, 512, 120), rng.integers(0, 512, 120))]
    check_entries(out, case.A[0], case.B[0], 512, 512, 512, 128, ents, 2)


def test_block_falls_back_when_several_blocks_are_needed(arb):
    """Column 35 of A is 2^900 larger than the rest: Algorithm 2 needs several blocks; the library
    then uses the classical algorithm, whose output matches the Algorithm 1 restatement."""
    rng = np.random.default_rng(4)
    M, K, N, p = 8, 70, 6, 64
    ea = rng.integers(-5, 5, size=M * K)
    ea[np.arange(M) * K + 35] += 900
    A = random_balls(rng, M * K, 1, 64, exps=ea)
    B = random_balls(rng, K * N, 1, 64, -5, 5)
    assert len(alg2.plan(A, B, M, K, N, p)[1]) > 1
    out, _ = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK)
    for i in range(M):
        for j in range(N):
            ref = alg1.matmul_entry(A, B, K, N, i, j, p, 1)
            idx = i * N + j
            got = ([int(out.limbs[0, idx])], int(out.exp[idx]), int(out.flags[idx]),
                   int(out.rad_man[idx]), int(out.rad_exp[idx]))
            assert got == (ref["limbs"], ref["exp"], ref["flags"], ref["rad_man"], ref["rad_exp"])


def test_identity_times_matrix(arb):
    """A * I = A when A has at most p bits (radius zero for exact A)."""
    rng = np.random.default_rng(8)
    n, p = 64, 128
    A = random_balls(rng, n * n, 2, 100, -30, 30)
    I = random_balls(rng, n * n, 1, 1, 1, 1)
    I.flags[:] = 2  # zero
    I.limbs[:] = 0
    I.exp[:] = 0
    d = np.arange(n) * n + np.arange(n)
    I.limbs[0, d] = np.uint64(1 << 63)
    I.exp[d] = 1
    I.flags[d] = 1 << 8
    out, _ = run_mm(arb, A, I, n, n, n, p, arb.ALG_BLOCK)
    for idx in range(0, n * n, 13):
        assert X.dy_cmp(X.mid(out, idx), X.mid(A, idx)) == 0
        assert int(out.rad_man[idx]) == 0
