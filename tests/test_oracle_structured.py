"""Structured inputs from the paper, on the oracle (CPU).

* Pascal matrices (Section V uses pi C(i+j, i)): with L the lower-triangular Pascal matrix
  L_ik = C(i, k), Vandermonde's identity gives (L L^T)_ij = C(i+j, i). So the exact product, the
  Algorithm 1 restatement and the Algorithm 2 restatement must all return that integer, with
  zero radius.
* The badly scaled 3 x 3 ball matrix of Section II, converted to binary balls outward. The
  classical algorithm keeps every entry of A A accurate to 2^-p of its own sum of magnitudes.
  Each entry's radius stays within twice its own propagated radius plus that rounding bound: the
  10^80 radius of the large entry does not spill into the small ones.
"""
from __future__ import annotations

from fractions import Fraction
from math import comb

import pytest

from oracle import alg1, alg2
from oracle import exact as X
from tests.ballmake import ball_values, make_balls
from tests.test_oracle_alg1 import out_mid_rad


def F(d):
    return X.dy_to_fraction(d)


def _pascal(n):
    L = [[comb(i, k) for k in range(n)] for i in range(n)]
    A = make_balls([L[i][k] for i in range(n) for k in range(n)])      # A = L, row-major
    B = make_balls([L[j][k] for k in range(n) for j in range(n)])      # B[k][j] = L[j][k]
    return A, B


def test_pascal_product_is_the_symmetric_pascal_matrix():
    n = 20
    A, B = _pascal(n)
    for i in range(n):
        for j in range(n):
            terms = X.matmul_entry_terms(A, B, n, n, i, j)
            m, r, _, _, _ = X.result_exact(terms, 64, 1)
            assert F(m) == comb(i + j, i) and r == (0, 0)
            if (i + j) % 7 == 0:  # the Algorithm 1 restatement on a sample of entries
                res = alg1.dot(alg1.real_terms(A, [i * n + k for k in range(n)], B,
                                               [k * n + j for k in range(n)]), 64, 1)
                mm, rr = out_mid_rad(res, 1)
                assert F(mm) == comb(i + j, i) and rr == (0, 0)


def test_pascal_product_through_scaled_integer_blocks():
    n = 40  # at least 30 indices, so Algorithm 2 forms a real block
    A, B = _pascal(n)
    h, blocks = alg2.plan(A, B, n, n, n, 64)
    C = [[Fraction(0)] * n for _ in range(n)]
    for start, stop, base in blocks:
        if base:
            for i in range(n):
                for j in range(n):
                    C[i][j] += sum(ball_values(A, i * n + k)[0] * ball_values(B, k * n + j)[0]
                                   for k in range(start, stop))
        else:
            e, f, Xs, Ys = alg2.scaled_block(A, B, n, n, n, start, stop)
            T = alg2.int_matmul(Xs, Ys)
            for i in range(n):
                for j in range(n):
                    C[i][j] += Fraction(T[i][j]) * Fraction(2) ** (-e[i] - f[j])
    assert any(not base for _, _, base in blocks)
    assert C == [[comb(i + j, i) for j in range(n)] for i in range(n)]


def _up30(x: Fraction) -> Fraction:
    """The least 30-bit binary value >= x > 0."""
    e = x.numerator.bit_length() - x.denominator.bit_length()
    while Fraction(2) ** e <= x:
        e += 1
    while Fraction(2) ** (e - 1) > x:
        e -= 1
    # 2^(e-1) <= x < 2^e: 30 significant bits at 2^(e-30)
    unit = Fraction(2) ** (e - 30)
    q = -((-x) // unit)  # ceil(x / unit)
    return q * unit


def _outward(mid: str, rad: str, bits: int):
    """A binary ball containing the decimal ball [mid +- rad]: the nearest `bits`-bit midpoint
    q 2^t (q an integer of at most `bits` bits), the radius plus the conversion error rounded up
    to 30 bits.  Returns (q, t, radius)."""
    v, r = Fraction(mid), Fraction(rad)
    if v == 0:
        return 0, 0, (_up30(r) if r else Fraction(0))
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e <= a:
        e += 1
    while Fraction(2) ** (e - 1) > a:
        e -= 1
    t = e - bits
    q = round(v / Fraction(2) ** t)
    err = abs(q * Fraction(2) ** t - v) + r
    return q, t, (_up30(err) if err else Fraction(0))


def _paper_matrix(nl):
    balls = [_outward(m, r, 64 * nl) for m, r in PAPER_3X3]
    A = make_balls([q for q, _, _ in balls], [r for _, _, r in balls], nlimbs=nl)
    for i, (q, t, _) in enumerate(balls):
        if q:
            A.exp[i] += t  # q 2^t
    for i, (m, r) in enumerate(PAPER_3X3):  # the binary ball contains the decimal one
        bm, br = ball_values(A, i)
        assert abs(bm - Fraction(m)) + Fraction(r) <= br
    return A


PAPER_3X3 = [("1.23e100", "1e80"), ("-1.5", "0"), ("0", "0"),
             ("1", "0"), ("2.34", "1e-20"), ("3.45", "1e-50"),
             ("0", "0"), ("2", "0"), ("4.56e-100", "1e-130")]


@pytest.mark.parametrize("prec", [64, 128, 256])
def test_badly_scaled_matrix_keeps_entrywise_accuracy(prec):
    nl = (prec + 63) // 64
    A = _paper_matrix(nl)
    n = 3
    for i in range(n):
        for j in range(n):
            xi, yi = [i * n + k for k in range(n)], [k * n + j for k in range(n)]
            S, Sabs, R = X.dot_terms_exact(X.real_dot_terms(A, xi, A, yi))
            res = alg1.dot(alg1.real_terms(A, xi, A, yi), prec, nl)
            m, r = out_mid_rad(res, nl)
            assert X.contains(m, r, S, R), (i, j)
            assert X.accuracy_ratio(m, S, Sabs, prec) <= 1.0, (i, j)
            bound = 2 * (F(R) + F(Sabs) * Fraction(2) ** -prec)
            assert F(r) <= bound, (i, j)  # the entry's own error scale, not the matrix's
    # no spill: C[2][2] = 2 * 3.45 + (4.56e-100)^2 keeps a radius at its own scale (the 2^-p
    # rounding of 6.9 and of the converted inputs), about 10^100 times below C[0][0]'s
    r22 = out_mid_rad(alg1.dot(alg1.real_terms(A, [6, 7, 8], A, [2, 5, 8]), prec, nl), nl)[1]
    r00 = out_mid_rad(alg1.dot(alg1.real_terms(A, [0, 1, 2], A, [0, 3, 6]), prec, nl), nl)[1]
    assert F(r22) < Fraction(1, 10 ** 15) and F(r00) > 10 ** 170
