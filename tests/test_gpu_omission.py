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
