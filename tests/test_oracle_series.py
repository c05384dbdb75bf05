"""Pins for the series exponential restatement (``oracle.series``, Section V's recurrence):
closed forms, sympy's independent Taylor expansion, the functional equation exp(f + g) =
exp(f) exp(g), and the propagated radius against exact evaluation at sampled points of the input
balls; planted slips in the recurrence must fail them."""
from __future__ import annotations

import math
import random
from fractions import Fraction

import pytest

from oracle import series as S


def _mul(p, q, n):
    return [sum(p[i] * q[k - i] for i in range(k + 1)) for k in range(n)]


def test_closed_forms():
    n = 20
    assert S.exp_series([0, 1], n) == [Fraction(1, math.factorial(k)) for k in range(n)]
    c = Fraction(-3, 7)
    assert S.exp_series([0, c], n) == [c ** k / math.factorial(k) for k in range(n)]
    b = S.exp_series([0, 0, 1], n)
    assert b == [Fraction(1, math.factorial(k // 2)) if k % 2 == 0 else 0 for k in range(n)]


def test_against_sympy_taylor_expansion():
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    a = [0, Fraction(1, 3), Fraction(-2, 5), Fraction(7, 4), Fraction(1, 9)]
    n = 12
    f = sum(sympy.Rational(v.numerator, v.denominator) * x ** j for j, v in enumerate(a))
    poly = sympy.series(sympy.exp(f), x, 0, n).removeO()
    want = [Fraction(int(sympy.fraction(c)[0]), int(sympy.fraction(c)[1]))
            for c in (poly.coeff(x, k) for k in range(n))]
    assert S.exp_series(a, n) == want


def test_functional_equation():
    rnd = random.Random(3)
    n = 15
    f = [0] + [Fraction(rnd.randint(-9, 9), rnd.randint(1, 9)) for _ in range(n - 1)]
    g = [0] + [Fraction(rnd.randint(-9, 9), rnd.randint(1, 9)) for _ in range(n - 1)]
    fg = [u + v for u, v in zip(f, g)]
    assert S.exp_series(fg, n) == _mul(S.exp_series(f, n), S.exp_series(g, n), n)


def test_propagated_radius_bounds_sampled_points():
    rnd = random.Random(5)
    n = 10
    a = [0] + [Fraction(rnd.randint(-50, 50), 16) for _ in range(n - 1)]
    rho = [0] + [Fraction(rnd.randint(0, 3), 1024) for _ in range(n - 1)]
    b, r = S.exp_series_radius(a, rho, n)
    for _ in range(30):
        pt = [0] + [a[j] + rho[j] * Fraction(rnd.randint(-100, 100), 100) for j in range(1, n)]
        bp = S.exp_series(pt, n)
        for k in range(n):
            assert abs(bp[k] - b[k]) <= r[k], k
    # the corner a_j + rho_j (all signs +) reaches close to the bound for positive coefficients
    pos = [0] + [abs(v) for v in a[1:]]
    _, rp = S.exp_series_radius(pos, rho, n)
    corner = S.exp_series([0] + [pos[j] + rho[j] for j in range(1, n)], n)
    base = S.exp_series(pos, n)
    assert all(corner[k] - base[k] == rp[k] for k in range(n))


def test_planted_slips_are_caught(monkeypatch):
    def wrong_weight(a, n):  # a_j instead of j a_j
        b = [Fraction(0)] * n
        b[0] = Fraction(1)
        for k in range(1, n):
            b[k] = sum(a[j] * b[k - j] for j in range(1, min(k, len(a) - 1) + 1)) / k
        return b

    def wrong_divisor(a, n):  # divided by k + 1
        b = [Fraction(0)] * n
        b[0] = Fraction(1)
        for k in range(1, n):
            b[k] = sum(j * a[j] * b[k - j] for j in range(1, min(k, len(a) - 1) + 1)) / (k + 1)
        return b
    for slip in (wrong_weight, wrong_divisor):
        monkeypatch.setattr(S, "exp_series", slip)
        with pytest.raises(AssertionError):
            test_closed_forms()
    monkeypatch.undo()
    test_closed_forms()
