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
from tests.gpu_util import env, to_raw

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
    assert any(n.startswith("digit_gemm") or n == "crt_gemm" for n in names)
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
    assert "crt_gemm" in names  # the multimodular engine is the default at this size
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


def check_bounds(out, A, B, M, K, N, prec, entries):
    """Containment and the accuracy bound |m - S| <= 2^-p sum |a b| for every listed entry."""
    worst = 0.0
    for i, j in entries:
        S, Sabs, R = X.dot_terms_exact(X.matmul_entry_terms(A, B, K, N, i, j))
        idx = i * N + j
        m, r = X.mid(out, idx), X.rad(out, idx)
        assert X.contains(m, r, S, R), (i, j)
        worst = max(worst, X.accuracy_ratio(m, S, Sabs, prec))
    assert worst <= 1.0, worst
    return worst


@pytest.fixture
def contiguous():
    """The inner index in its own order (the inner ordering of Section IV-B off) and every input
    bit kept (no negligible-limb omission), so that the blocks are the contiguous ones of
    ``alg2.plan``."""
    with env(ARBGPU_INNER_ORDER="0", ARBGPU_OMIT="0"):
        yield


def jump_case(seed, M, K, N, jumps, p, nl=1, rad=None):
    """Columns listed in `jumps` of A are 2^900 larger than the rest: Algorithm 2 cuts there."""
    rng = np.random.default_rng(seed)
    ea = rng.integers(-5, 5, size=M * K)
    for k in jumps:
        ea[np.arange(M) * K + k] += 900
    A = random_balls(rng, M * K, nl, 64 * nl, exps=ea, rad_bits=rad, rad_zero_frac=0.5)
    B = random_balls(rng, K * N, nl, 64 * nl, -5, 5, rad_bits=rad, rad_zero_frac=0.5)
    return A, B


def band_case(seed, M, K, N, lo, hi, nl=1, rad=None):
    """Columns lo..hi-1 of A are 2^900 larger than the rest: three full blocks."""
    rng = np.random.default_rng(seed)
    ea = rng.integers(-5, 5, size=M * K)
    for k in range(lo, hi):
        ea[np.arange(M) * K + k] += 900
    A = random_balls(rng, M * K, nl, 64 * nl, exps=ea, rad_bits=rad, rad_zero_frac=0.5)
    B = random_balls(rng, K * N, nl, 64 * nl, -5, 5, rad_bits=rad, rad_zero_frac=0.5)
    return A, B


def test_several_blocks_with_basecase(arb, contiguous):
    """Column 35 of A jumps by 2^900: blocks [0, 35), a one-column block widened to a 30-column
    basecase, then the rest; the block part is accumulated and the basecase done by dots."""
    M, K, N, p = 24, 100, 20, 64
    A, B = jump_case(4, M, K, N, [35], p, rad=60)
    h, blocks = alg2.plan(A, B, M, K, N, p)
    assert any(b[2] for b in blocks) and any(not b[2] for b in blocks)
    out, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "accumulate" in names and "plan" in names
    assert "dot_tile" in names or "dot_fused" in names  # (tiles only when they fill the SMs)
    check_bounds(out, A, B, M, K, N, p, [(i, j) for i in range(M) for j in range(N)])


def test_several_blocks_without_basecase(arb, contiguous):
    """Columns 60..119 of A sit 2^900 higher: three full blocks, no basecase."""
    M, K, N, p = 40, 180, 36, 128
    A, B = band_case(5, M, K, N, 60, 120, nl=2, rad=120)
    h, blocks = alg2.plan(A, B, M, K, N, p)
    assert len(blocks) >= 3 and not any(b[2] for b in blocks)
    out, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "acc_round" in names and "dot_tile" not in names and "dot_fused" not in names
    assert names.count("accumulate") == len(blocks)
    rng = np.random.default_rng(2)
    check_bounds(out, A, B, M, K, N, p, [(int(a), int(b)) for a, b in
                                         zip(rng.integers(0, M, 200), rng.integers(0, N, 200))])


def test_structured_laplace_blocks(arb, contiguous):
    """Exponents c_k + U[-4, 4] with c_k ~ Laplace(40) along the inner index (the structured complex
    workload's real part at a small size): many blocks of the plan, exact accumulation, bounds."""
    rng = np.random.default_rng(7)
    n, p = 160, 128
    c = np.clip(np.rint(rng.laplace(0, 40, size=n)), -200, 200).astype(np.int64)
    ea = np.clip(c[None, :] + rng.integers(-4, 4, size=(n, n), endpoint=True), -200, 200)
    eb = np.clip(c[:, None] + rng.integers(-4, 4, size=(n, n), endpoint=True), -200, 200)
    A = random_balls(rng, n * n, 2, 128, exps=ea.reshape(-1), rad_bits=120)
    B = random_balls(rng, n * n, 2, 128, exps=eb.reshape(-1), rad_bits=120)
    h, blocks = alg2.plan(A, B, n, n, n, p)
    assert len(blocks) >= 2
    out, names = run_mm(arb, A, B, n, n, n, p, arb.ALG_BLOCK, trace=True)
    assert "plan" in names
    # one accumulation per full block of the oracle's plan: the device planner agrees with it
    assert names.count("accumulate") == sum(1 for b in blocks if not b[2])
    rng2 = np.random.default_rng(3)
    check_bounds(out, A, B, n, n, n, p, [(int(a), int(b)) for a, b in
                                         zip(rng2.integers(0, n, 150), rng2.integers(0, n, 150))])


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


def run_cmm(arb, A2, B2, M, K, N, prec, alg, trace=False, flags=0):
    nl = (prec + 63) // 64
    ctx = arb.default_context()
    C2 = [arb.Balls.empty(M * N, nl), arb.Balls.empty(M * N, nl)]
    if trace:
        ctx.trace(True)
    arb.mat_mul(C2, [arb.Balls.from_raw(a) for a in A2], [arb.Balls.from_raw(b) for b in B2], M, K,
                N, prec, alg=alg, flags=flags)
    st = ctx.status()
    names = [r[0] for r in ctx.trace_read()] if trace else []
    ctx.trace(False)
    assert st == 0
    return [to_raw(c) for c in C2], names


def check_complex(outs, A2, B2, M, K, N, prec, entries):
    worst = 0.0
    for i, j in entries:
        re, im = X.complex_dot_terms(A2, [i * K + k for k in range(K)], B2,
                                     [k * N + j for k in range(K)])
        for part, terms in ((0, re), (1, im)):
            S, Sabs, R = X.dot_terms_exact(terms)
            idx = i * N + j
            m, r = X.mid(outs[part], idx), X.rad(outs[part], idx)
            assert X.contains(m, r, S, R), (part, i, j)
            worst = max(worst, X.accuracy_ratio(m, S, Sabs, prec))
    assert worst <= 1.0, worst


def test_complex_block_uniform(arb):
    """Uniformly scaled complex matrices: four single-block real products, Re = ArBr - AiBi and
    Im = ArBi + AiBr accumulated exactly (Section IV-C)."""
    rng = np.random.default_rng(21)
    n, p = 96, 128
    A2 = [random_balls(rng, n * n, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5) for _ in "ri"]
    B2 = [random_balls(rng, n * n, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5) for _ in "ri"]
    outs, names = run_cmm(arb, A2, B2, n, n, n, p, arb.ALG_BLOCK, trace=True)
    assert names.count("accumulate") == 4
    assert "crt_gemm" in names or "digit_gemm_mid" in names
    rng2 = np.random.default_rng(4)
    check_complex(outs, A2, B2, n, n, n, p, [(int(a), int(b)) for a, b in
                                             zip(rng2.integers(0, n, 80), rng2.integers(0, n, 80))])


@pytest.mark.parametrize("M,K,N,prec,spread", [(96, 96, 96, 128, 10), (70, 100, 90, 256, 20),
                                                (33, 200, 130, 64, 3)])
def test_complex_3m_exact_rounding(arb, M, K, N, prec, spread):
    """Eq. 2 (Section IV-C): with one scaling per row of A and column of B shared by both parts,
    Re = P1 - P2 and Im = P3 - P1 - P2 from three exact products.  The integers are exact, so
    every sampled midpoint is RNE_p of the exact part, the same as the four-product path gives,
    and every ball contains the exact value."""
    rng = np.random.default_rng(60 + M)
    nl = (prec + 63) // 64
    A2 = [random_balls(rng, M * K, nl, prec, -spread, spread, rad_bits=prec - 8,
                       rad_zero_frac=0.5) for _ in "ri"]
    B2 = [random_balls(rng, K * N, nl, prec, -spread, spread, rad_bits=prec - 8,
                       rad_zero_frac=0.5) for _ in "ri"]
    o3, n3 = run_cmm(arb, A2, B2, M, K, N, prec, arb.ALG_BLOCK, trace=True,
                     flags=arb.MM_COMPLEX_3M)
    assert "z3m" in n3 and "residue_sum" in n3
    assert n3.count("crt_gemm") == 1 and n3.count("residues") == 2
    o4, n4 = run_cmm(arb, A2, B2, M, K, N, prec, arb.ALG_BLOCK, trace=True)
    assert "z3m" not in n4
    for a, b in zip(o3, o4):
        for f in ("limbs", "exp", "flags"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
    rng2 = np.random.default_rng(6)
    entries = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 40), rng2.integers(0, N, 40))]
    check_complex(o3, A2, B2, M, K, N, prec, entries)
    for i, j in entries:
        re, im = X.complex_dot_terms(A2, [i * K + k for k in range(K)], B2,
                                     [k * N + j for k in range(K)])
        idx = i * N + j
        for part, terms in ((0, re), (1, im)):
            m_ref = X.result_exact(terms, prec, nl)[0]
            limbs, e, fl = X.encode_mid(m_ref, nl)
            got = ([int(o3[part].limbs[k, idx]) for k in range(nl)], int(o3[part].exp[idx]),
                   int(o3[part].flags[idx]))
            assert got == (limbs, e, fl), (part, i, j)


def test_complex_3m_exact_inputs_and_zero_part(arb):
    """Eq. 2 with exact inputs whose imaginary parts are zero in A: Im C = Ar Bi exactly, zero
    radii wherever the exact sums fit in p bits (small integers)."""
    rng = np.random.default_rng(70)
    M, K, N, p = 64, 64, 64, 128
    A2 = [random_balls(rng, M * K, 2, 8, 8, 8) for _ in "ri"]
    B2 = [random_balls(rng, K * N, 2, 8, 8, 8) for _ in "ri"]
    A2[1].flags[:] = 2
    A2[1].limbs[:] = 0
    A2[1].exp[:] = 0
    o3, n3 = run_cmm(arb, A2, B2, M, K, N, p, arb.ALG_BLOCK, trace=True, flags=arb.MM_COMPLEX_3M)
    assert "z3m" in n3
    for idx in range(0, M * N, 37):
        for part in (0, 1):
            assert int(o3[part].rad_man[idx]) == 0
    rng2 = np.random.default_rng(7)
    check_complex(o3, A2, B2, M, K, N, p,
                  [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 30), rng2.integers(0, N, 30))])


def test_complex_3m_plans_several_blocks_for_both_parts(arb, contiguous):
    """When the shared scaling needs several blocks (Laplace exponents along the inner index), the
    flag cuts the inner range once for both parts (Section IV-C's second suggestion): one plan
    record, the greedy blocks of the merged entry heights (here every block is a basecase range of
    complex dots), and the result is still rigorous."""
    from synth.workloads import complex_matmul_laplace
    case = complex_matmul_laplace(n=128, structured=True)
    outs, names = run_cmm(arb, case.A, case.B, 128, 128, 128, 128, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    h, blocks = alg2.plan_complex_shared(case.A, case.B, 128, 128, 128, 128)
    assert arb.default_context().last_plans() == [dict(kind=2, h=h, K=128, blocks=blocks)]
    assert len(blocks) > 1 and "plan" in names
    rng2 = np.random.default_rng(8)
    check_complex(outs, case.A, case.B, 128, 128, 128, 128,
                  [(int(a), int(b)) for a, b in zip(rng2.integers(0, 128, 30),
                                                    rng2.integers(0, 128, 30))])


@pytest.mark.parametrize("structured", [True, False])
def test_complex_laplace_small(arb, contiguous, structured):
    """The complex Laplace(40) workload at N = 128: structured (blocks along the inner index) and
    literal (i.i.d. exponents: mostly basecase blocks)."""
    from synth.workloads import complex_matmul_laplace
    case = complex_matmul_laplace(n=128, structured=structured)
    outs, names = run_cmm(arb, case.A, case.B, 128, 128, 128, 128, arb.ALG_BLOCK, trace=True)
    assert "plan" in names
    rng2 = np.random.default_rng(5)
    check_complex(outs, case.A, case.B, 128, 128, 128, 128,
                  [(int(a), int(b)) for a, b in zip(rng2.integers(0, 128, 60),
                                                    rng2.integers(0, 128, 60))])


def _run_engine(arb, engine, A, B, M, K, N, prec, cplx=False):
    # (the omission of negligible limbs always takes the multimodular engine: kept off here)
    with env(ARBGPU_ENGINE=engine, ARBGPU_OMIT="0"):
        if cplx:
            outs, names = run_cmm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, trace=True)
        else:
            out, names = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, trace=True)
            outs = [out]
    return outs, names


@pytest.mark.parametrize("kind", ["single", "several", "complex", "p512"])
def test_digit_and_multimodular_engines_agree_bit_for_bit(arb, kind):
    """The exact block integers T are the same whichever engine forms them (digit products or
    residues + Chinese remainder theorem), so every output field must agree."""
    rng = np.random.default_rng(40)
    if kind == "single":
        M, K, N, p = 130, 192, 120, 256
        A = random_balls(rng, M * K, 4, 256, -20, 20, rad_bits=250, rad_zero_frac=0.3)
        B = random_balls(rng, K * N, 4, 256, -20, 20, rad_bits=250, rad_zero_frac=0.3)
    elif kind == "p512":  # about 100 moduli, 28 32-bit chunks per scaled integer
        M, K, N, p = 67, 100, 45, 512
        A = random_balls(rng, M * K, 8, 512, -20, 20, rad_bits=500, rad_zero_frac=0.3)
        B = random_balls(rng, K * N, 8, 512, -20, 20, rad_bits=500, rad_zero_frac=0.3)
    elif kind == "several":
        M, K, N, p = 40, 180, 36, 128
        A, B = band_case(5, M, K, N, 60, 120, nl=2, rad=120)
    else:
        M = K = N = 80
        p = 128
        A = [random_balls(rng, M * K, 2, 128, -10, 10, rad_bits=120) for _ in "ri"]
        B = [random_balls(rng, K * N, 2, 128, -10, 10, rad_bits=120) for _ in "ri"]
    od, nd = _run_engine(arb, "digits", A, B, M, K, N, p, cplx=(kind == "complex"))
    oc, nc = _run_engine(arb, "crt", A, B, M, K, N, p, cplx=(kind == "complex"))
    assert "crt_gemm" in nc and "crt_gemm" not in nd
    for a, b in zip(od, oc):
        for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_multimodular_p1024(arb):
    """p = 1024: 1024-bit mantissas, about 190 moduli; midpoints are the exactly rounded values."""
    rng = np.random.default_rng(41)
    M, K, N, p = 48, 64, 40, 1024
    A = random_balls(rng, M * K, 16, 1024, -50, 50, rad_bits=1016, rad_zero_frac=0.5)
    B = random_balls(rng, K * N, 16, 1024, -50, 50, rad_bits=1016, rad_zero_frac=0.5)
    rng2 = np.random.default_rng(2)
    sample = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 40), rng2.integers(0, N, 40))]
    for engine, kernel in (("crt", "crt_gemm"), ("digits", "digit_gemm_mid")):
        (out,), names = _run_engine(arb, engine, A, B, M, K, N, p)
        assert kernel in names
        check_entries(out, A, B, M, K, N, p, sample, 16)


def test_multimodular_kp_1024_one_chain(arb):
    """K = 1000 (Kp = 1024): the residue products' longest single chain, whose quarter sums reach
    2^24, reduced modulo m in FP32 by the GEMM's drain; midpoints exactly rounded."""
    rng = np.random.default_rng(44)
    M, K, N, p = 40, 1000, 36, 128
    A = random_balls(rng, M * K, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5)
    B = random_balls(rng, K * N, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5)
    (out,), names = _run_engine(arb, "crt", A, B, M, K, N, p)
    assert "crt_gemm" in names
    (dig,), _ = _run_engine(arb, "digits", A, B, M, K, N, p)
    for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
        assert np.array_equal(getattr(out, f), getattr(dig, f)), f
    rng2 = np.random.default_rng(5)
    check_entries(out, A, B, M, K, N, p, [(int(a), int(b)) for a, b in
                                         zip(rng2.integers(0, M, 30), rng2.integers(0, N, 30))], 2)


def test_multimodular_long_inner_dimension(arb):
    """K > 1024: the residue products run in the general GEMM's multimodular mode (chains of at
    most 256 products, carries between them); midpoints are still the exactly rounded values."""
    rng = np.random.default_rng(43)
    M, K, N, p = 40, 1100, 36, 128
    A = random_balls(rng, M * K, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5)
    B = random_balls(rng, K * N, 2, 128, -10, 10, rad_bits=120, rad_zero_frac=0.5)
    (out,), names = _run_engine(arb, "crt", A, B, M, K, N, p)
    assert "crt_gemm" in names
    rng2 = np.random.default_rng(4)
    check_entries(out, A, B, M, K, N, p, [(int(a), int(b)) for a, b in
                                         zip(rng2.integers(0, M, 30), rng2.integers(0, N, 30))], 2)


def _balls_of(values, nl):
    """Raw balls of exact dyadic values (num, exp) with zero radii."""
    from synth import RawBalls
    r = RawBalls.zeros(len(values), nl)
    for q, v in enumerate(values):
        limbs, e, fl = X.encode_mid(v, nl)
        for k in range(nl):
            r.limbs[k, q] = np.uint64(limbs[k])
        r.exp[q] = e
        r.flags[q] = fl
    return r


@pytest.mark.parametrize("tail", [1, -1, 0])
def test_tie_broken_below_the_rounding_window(arb, tail):
    """Each entry is (2^128 + 1) * 1 + tail * 2^-200 * 2^-200: a tie at p = 128 that only the term
    2^-400, 529 bits below the top, decides -- below the 6-limb window of |T| that the
    multimodular epilogue rounds.  The midpoint must be RNE_128 of the exact sum (up, down, or to
    even without the term) and the ball must contain it."""
    M, K, N, p = 4, 48, 4, 128
    nl = 3
    zero = (0, 0)
    a = [zero] * (M * K)
    b = [zero] * (K * N)
    for i in range(M):
        a[i * K] = ((1 << 128) + 1, 0)
        if tail:
            a[i * K + 1] = (1, -200)
    for j in range(N):
        b[j] = (1, 0)
        if tail:
            b[N + j] = (tail, -200)
    A, B = _balls_of(a, nl), _balls_of(b, nl)
    (out,), names = _run_engine(arb, "crt", A, B, M, K, N, p)
    assert "crt_gemm" in names
    check_entries(out, A, B, M, K, N, p, [(i, j) for i in range(M) for j in range(N)], 2)


def test_pascal_product_closed_form(arb):
    """L L^T = C(i+j, i) for the lower-triangular Pascal matrix L_ik = C(i, k) (Vandermonde's
    identity; Section V multiplies Pascal matrices): exact integers up to C(126, 63) < 2^122, so
    at p = 128 every entry is exact with zero radius, through one scaled integer block."""
    from math import comb
    from tests.ballmake import make_balls
    n, p = 64, 128
    A = make_balls([comb(i, k) for i in range(n) for k in range(n)])
    B = make_balls([comb(j, k) for k in range(n) for j in range(n)])
    out, names = run_mm(arb, A, B, n, n, n, p, arb.ALG_BLOCK, nl_out=2, trace=True)
    assert "plan" not in names  # one block
    for i in range(n):
        for j in range(n):
            idx = i * n + j
            assert X.dy_to_fraction(X.mid(out, idx)) == comb(i + j, i), (i, j)
            assert int(out.rad_man[idx]) == 0, (i, j)


@pytest.mark.parametrize("cplx", [False, True])
def test_basecase_dots_tiled_equal_lane_groups(arb, cplx):
    """The basecase blocks of Algorithm 2 through the tiled dot kernel equal, in every output
    field, the group-of-lanes kernel (ARBGPU_DOT_TILE=0): the tagged index lists, the complex
    combinations and the accumulated blocks as `initial` term."""
    from synth.workloads import complex_matmul_laplace
    if cplx:  # tiles of 32 x 32 entries: enough of them to fill the SMs
        case = complex_matmul_laplace(n=448, structured=False)
        A, B, M, K, N, p = case.A, case.B, 448, 448, 448, 128
    else:
        A, B = jump_case(4, 640, 100, 320, [35], 64, rad=60)
        M, K, N, p = 640, 100, 320, 64
    outs = []
    for tile in ("1", "0"):
        # every input bit kept, so that basecase blocks remain
        with env(ARBGPU_DOT_TILE=tile, ARBGPU_OMIT="0"):
            if cplx:
                o, names = run_cmm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
            else:
                o1, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
                o = [o1]
            assert ("dot_tile" in names) == (tile == "1")
            outs.append(o)
    for a, b in zip(outs[0], outs[1]):
        for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
