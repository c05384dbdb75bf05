"""Negligible-limb omission in Algorithm 2 (Section IV-B's last paragraph, in the reading of
``oracle.alg2.omission_thresholds``) on the GPU: when some line is much taller than the precision
needs, the bits below each line's threshold are dropped and the product runs as one block.  The
midpoints must then be exactly RNE_p of the oracle's product of the truncated operands, and every
ball must contain the exact product within the accuracy bound 2^-p sum |a b|."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import alg2
from oracle import exact as X
from synth import random_balls
from tests.gpu_util import env, to_raw
from tests.test_gpu_block import check_bounds, check_complex, run_cmm, run_mm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def _rne(v, p, nl):
    from fractions import Fraction
    num, den = v.numerator, v.denominator
    # the dyadic value of a Fraction whose denominator is a power of two
    e = -(den.bit_length() - 1) if den > 1 else 0
    assert Fraction(num) * Fraction(2) ** e == v
    return X.encode_mid(X.rne((num, e), p)[0], nl)


@pytest.mark.parametrize("M,K,N,p,bits,spread", [(40, 40, 36, 64, 1024, 5),
                                                  (33, 60, 30, 128, 256, 200)])
def test_omitted_single_block_is_rne_of_the_truncated_product(arb, M, K, N, p, bits, spread):
    rng = np.random.default_rng(M + K + N + p)
    nl = (bits + 63) // 64
    A = random_balls(rng, M * K, nl, bits, -spread, spread, rad_bits=bits - 4,
                     rad_zero_frac=0.5)
    B = random_balls(rng, K * N, nl, bits, -spread, spread, rad_bits=bits - 4,
                     rad_zero_frac=0.5)
    h, blocks = alg2.plan(A, B, M, K, N, p)
    assert blocks != [(0, K, False)]  # several blocks without the omission
    out, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "omission" in names and "plan" not in names
    assert arb.default_context().last_plans() == [dict(kind=3, h=h, K=K, blocks=[(0, K, False)])]
    tau, sigma = alg2.omission_thresholds(A, B, M, K, N, p)
    T = alg2.omitted_product(A, B, M, K, N, tau, sigma)
    onl = (p + 63) // 64
    rng2 = np.random.default_rng(3)
    ents = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 60), rng2.integers(0, N, 60))]
    for i, j in ents:
        idx = i * N + j
        got = ([int(out.limbs[k, idx]) for k in range(onl)], int(out.exp[idx]),
               int(out.flags[idx]))
        assert got == _rne(T[i][j], p, onl), (i, j)
    check_bounds(out, A, B, M, K, N, p, ents)


def test_omitted_complex_product(arb):
    """A complex product of 1024-bit entries at p = 64: each of the four real products runs as one
    block of truncated operands and is accumulated into its part; every checked ball contains the
    exact product within the bound."""
    rng = np.random.default_rng(31)
    n, p = 48, 64
    A2 = [random_balls(rng, n * n, 16, 1024, -6, 6, rad_bits=1000, rad_zero_frac=0.5)
          for _ in "ri"]
    B2 = [random_balls(rng, n * n, 16, 1024, -6, 6, rad_bits=1000, rad_zero_frac=0.5)
          for _ in "ri"]
    outs, names = run_cmm(arb, A2, B2, n, n, n, p, arb.ALG_BLOCK, trace=True)
    plans = arb.default_context().last_plans()
    assert len(plans) == 4 and all(r["kind"] == 3 for r in plans)
    assert "dot_tile" not in names and "dot_fused" not in names
    rng2 = np.random.default_rng(9)
    check_complex(outs, A2, B2, n, n, n, p, [(int(a), int(b)) for a, b in
                                             zip(rng2.integers(0, n, 50), rng2.integers(0, n, 50))])


def test_omission_off_keeps_every_bit(arb):
    """ARBGPU_OMIT=0: the same product runs over its blocks, untruncated; both results contain the
    exact product within the bound."""
    rng = np.random.default_rng(12)
    M, K, N, p = 30, 48, 20, 64
    A = random_balls(rng, M * K, 16, 1024, -5, 5)
    B = random_balls(rng, K * N, 16, 1024, -5, 5)
    ents = [(i, j) for i in range(0, M, 3) for j in range(0, N, 3)]
    with env(ARBGPU_OMIT="0"):
        off, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "omission" not in names
    on, names = run_mm(arb, A, B, M, K, N, p, arb.ALG_BLOCK, trace=True)
    assert "omission" in names
    check_bounds(off, A, B, M, K, N, p, ents)
    check_bounds(on, A, B, M, K, N, p, ents)


# ---- eq. 2 with the omission under thresholds shared by both parts
# (``oracle.alg2.omission_thresholds_complex``)

def _eq2_case(kind):
    from synth.workloads import complex_matmul_laplace
    if kind == "wide":  # 1024-bit entries at p = 64
        rng = np.random.default_rng(31)
        n, p = 40, 64
        mk = lambda: random_balls(rng, n * n, 16, 1024, -6, 6, rad_bits=1000,  # noqa
                                  rad_zero_frac=0.5)
        return [mk(), mk()], [mk(), mk()], n, p
    if kind == "lopsided":  # A_re and B_im 2^200 below A_im and B_re: Re ~ 2^-200 Im
        rng = np.random.default_rng(32)
        n, p = 36, 128

        def mk(low):
            d = -200 if low else 0
            return random_balls(rng, n * n, 8, 512, -5 + d, 5 + d, rad_bits=500,
                                rad_zero_frac=0.5)
        return [mk(True), mk(False)], [mk(False), mk(True)], n, p
    case = complex_matmul_laplace(n=64, structured=(kind == "laplace"))
    return case.A, case.B, 64, case.prec


def _truncated_part(A2, B2, K, N, tau, sigma, part, i, j):
    """Part `part` of entry (i, j) of the exact complex product of the truncated operands."""
    from fractions import Fraction

    def val(raw, idx, t):
        v, e = alg2.truncate_value(alg2.top_bottom(raw, idx), t)
        return Fraction(v) * Fraction(2) ** e
    pairs = (((0, 0, 1), (1, 1, -1)), ((0, 1, 1), (1, 0, 1)))[part]
    return sum(sg * val(A2[x], i * K + k, tau[i]) * val(B2[y], k * N + j, sigma[j])
               for x, y, sg in pairs for k in range(K))


@pytest.mark.parametrize("kind", ["wide", "lopsided", "laplace"])
def test_eq2_omitted_single_block_is_rne_of_the_truncated_product(arb, kind):
    """Eq. 2 with ARBGPU_MM_COMPLEX_3M where the parts' shared scaling needs several blocks: both
    parts drop their bits below thresholds shared by the parts and the truncated parts form one
    shared block (record kind 5), so every sampled midpoint of Re and Im is exactly RNE_p of the
    oracle's truncated complex product, and every ball contains the exact product within the
    accuracy bound (per part: the lopsided case fails it if the thresholds follow the larger
    part's bound alone)."""
    A2, B2, n, p = _eq2_case(kind)
    h, blocks = alg2.plan_complex_shared(A2, B2, n, n, n, p)
    assert len(blocks) > 1  # several shared blocks without the omission
    outs, names = run_cmm(arb, A2, B2, n, n, n, p, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    assert "omission" in names and "z3m" in names and "plan" not in names
    assert arb.default_context().last_plans() == [dict(kind=5, h=h, K=n,
                                                       blocks=[(0, n, False)])]
    tau, sigma = alg2.omission_thresholds_complex(A2, B2, n, n, n, p)
    onl = (p + 63) // 64
    rng2 = np.random.default_rng(5)
    ents = [(int(a), int(b)) for a, b in zip(rng2.integers(0, n, 40), rng2.integers(0, n, 40))]
    for i, j in ents:
        idx = i * n + j
        for part in (0, 1):
            T = _truncated_part(A2, B2, n, n, tau, sigma, part, i, j)
            out = outs[part]
            got = ([int(out.limbs[k, idx]) for k in range(onl)], int(out.exp[idx]),
                   int(out.flags[idx]))
            assert got == _rne(T, p, onl), (kind, part, i, j)
    check_complex(outs, A2, B2, n, n, n, p, ents)


def test_eq2_falls_back_to_four_products_when_the_shared_omission_leaves_several_blocks(arb):
    """The literal Laplace workload at N = 64: thresholds shared by the parts leave rows taller
    than h, so the flag runs four real products, each with its own omission; the balls stay
    rigorous."""
    A2, B2, n, p = _eq2_case("laplace_literal")
    outs, names = run_cmm(arb, A2, B2, n, n, n, p, arb.ALG_BLOCK, trace=True,
                          flags=arb.MM_COMPLEX_3M)
    plans = arb.default_context().last_plans()
    assert len(plans) == 4 and "z3m" not in names
    rng2 = np.random.default_rng(6)
    check_complex(outs, A2, B2, n, n, n, p, [(int(a), int(b)) for a, b in
                                             zip(rng2.integers(0, n, 40), rng2.integers(0, n, 40))])


# ---- the max-plus bound on 16-bit halves (maxplus16_top_kernel) against the int32 kernel

def _wide_rows_case():
    """Complex 512-bit entries at p = 64 whose rows of A span more than 2^13 bits of exponent
    (column 0 sits 2^9000 above the rest): the int32 max-plus kernel runs there."""
    rng = np.random.default_rng(77)
    n, p = 40, 64
    A2, B2 = [], []
    for _ in "ri":
        ea = rng.integers(-6, 6, size=n * n)
        ea[np.arange(n) * n] += 9000
        A2.append(random_balls(rng, n * n, 8, 512, exps=ea, rad_bits=500, rad_zero_frac=0.5))
        B2.append(random_balls(rng, n * n, 8, 512, -6, 6, rad_bits=500, rad_zero_frac=0.5))
    return A2, B2, n, p


@pytest.mark.parametrize("kind,m3", [("laplace", False), ("laplace", True),
                                     ("laplace_literal", True), ("lopsided", True),
                                     ("wide_rows", False)])
def test_maxplus16_gives_the_int32_results(arb, kind, m3):
    """The window bound and the omission thresholds from the 16-bit max-plus kernel equal those of
    the int32 kernel wherever a product is nonzero, so every output field is bit-identical with
    ARBGPU_MAXPLUS16=0; rows wider than 2^13 bits take the int32 kernel (and the balls stay
    rigorous)."""
    from tests.gpu_util import env
    A2, B2, n, p = _wide_rows_case() if kind == "wide_rows" else _eq2_case(kind)
    flags = arb.MM_COMPLEX_3M if m3 else 0
    runs = []
    for v in ("1", "0"):
        with env(ARBGPU_MAXPLUS16=v):
            outs, names = run_cmm(arb, A2, B2, n, n, n, p, arb.ALG_BLOCK, trace=True, flags=flags)
        assert "maxplus_top" in names
        runs.append(outs)
    for a, b in zip(*runs):
        for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), (kind, f)
    rng2 = np.random.default_rng(12)
    check_complex(runs[0], A2, B2, n, n, n, p, [(int(a), int(b)) for a, b in
                                                zip(rng2.integers(0, n, 30),
                                                    rng2.integers(0, n, 30))])
