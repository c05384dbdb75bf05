"""Pins for the exact oracle (``oracle.exact``) against things other than itself: Python's float
semantics, ``fractions.Fraction`` arithmetic, mpmath's correctly rounded conversion, hand-made
values and closed forms."""
from __future__ import annotations

import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X
from synth import FLAG_NAN, RawBalls, random_balls
from tests.ballmake import ball_values, make_balls


def F(d):
    return X.dy_to_fraction(d)


def test_decode_matches_float_semantics():
    """Layout built from math.frexp of doubles decodes to exactly Fraction(double)."""
    rng = random.Random(1)
    vals = [rng.uniform(-1e6, 1e6) * 2.0 ** rng.randint(-300, 300) for _ in range(200)] + [1.0,
                                                                                             -0.375]
    raw = RawBalls.zeros(len(vals), 1)
    for i, v in enumerate(vals):
        f, e = math.frexp(v)
        raw.limbs[0, i] = np.uint64(int(abs(f) * 2**53) << 11)
        raw.exp[i] = e
        raw.flags[i] = (1 if v < 0 else 0) | (1 << 8)
    for i, v in enumerate(vals):
        assert F(X.mid(raw, i)) == Fraction(v)


def test_decode_handmade_multilimb():
    raw = make_balls([Fraction(3, 8), Fraction(-5), Fraction(7, 2**70)],
                     nlimbs=2)
    assert F(X.mid(raw, 0)) == Fraction(3, 8)
    assert F(X.mid(raw, 1)) == -5
    assert F(X.mid(raw, 2)) == Fraction(7, 2**70)
    # 0.375 = 0.75 * 2^-1: top limb 0xC000..., exponent -1
    assert int(raw.limbs[1, 0]) == 0xC000000000000000 and int(raw.exp[0]) == -1


@pytest.mark.parametrize("seed", range(5))
def test_exact_dot_vs_fraction_bruteforce(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 6)
    xs = [Fraction(rng.randint(-2**40, 2**40), 2**rng.randint(0, 90)) for _ in range(n)]
    ys = [Fraction(rng.randint(-2**40, 2**40), 2**rng.randint(0, 90)) for _ in range(n)]
    rx = [Fraction(rng.randint(0, 2**20), 2**rng.randint(20, 60)) for _ in range(n)]
    ry = [Fraction(rng.randint(0, 2**20), 2**rng.randint(20, 60)) for _ in range(n)]
    xr = make_balls(xs, rx, nlimbs=1)
    yr = make_balls(ys, ry, nlimbs=1)
    sub = seed % 2 == 1
    terms = X.real_dot_terms(xr, range(n), yr, range(n), sub=sub)
    init = (Fraction(rng.randint(-99, 99), 8), Fraction(1, 2**10))
    ib = make_balls([init[0]], [init[1]])
    S, Sabs, R = X.dot_terms_exact(terms, X.ball(ib, 0))
    sgn = -1 if sub else 1
    assert F(S) == init[0] + sgn * sum(a * b for a, b in zip(xs, ys))
    assert F(Sabs) == abs(init[0]) + sum(abs(a * b) for a, b in zip(xs, ys))
    assert F(R) == init[1] + sum(abs(a) * s + abs(b) * r + r * s
                                 for a, b, r, s in zip(xs, ys, rx, ry))


def test_complex_terms_closed_form():
    a, b, c, d = Fraction(3, 4), Fraction(-5, 8), Fraction(7, 2), Fraction(1, 16)
    xr, xi = make_balls([a]), make_balls([b])
    yr, yi = make_balls([c]), make_balls([d])
    re, im = X.complex_dot_terms((xr, xi), [0], (yr, yi), [0])
    assert F(X.dot_terms_exact(re)[0]) == a * c - b * d
    assert F(X.dot_terms_exact(im)[0]) == a * d + b * c


def _random_dyadic(rng, bits):
    return (rng.randint(-(2**bits), 2**bits), rng.randint(-200, 200))


def test_rne_matches_float_at_53_bits():
    """float(Fraction) is correctly rounded to nearest-even at 53 bits."""
    rng = random.Random(7)
    cases = [_random_dyadic(rng, rng.randint(54, 200)) for _ in range(3000)]
    # ties: exactly half an ulp above an even and an odd 53-bit integer
    cases += [((1 << 60) + (1 << 7), 0), ((1 << 60) + (3 << 7), 0), (-((1 << 60) + (1 << 7)), 0)]
    for v in cases:
        r, err = X.rne(v, 53)
        assert F(r) == Fraction(float(F(v)))
        assert F(err) == abs(F(r) - F(v))


@pytest.mark.parametrize("p", [2, 3, 63, 64, 65, 128, 192, 256, 1024])
def test_rne_matches_mpmath(p):
    """mpmath's own round-to-nearest-even of a dyadic (``libmp.from_man_exp`` with rounding 'n')."""
    mpmath = pytest.importorskip("mpmath")
    libmp = mpmath.libmp
    rng = random.Random(p)
    for _ in range(400):
        v = _random_dyadic(rng, rng.randint(1, p + 80))
        r, _ = X.rne(v, p)
        sign, man, exp, _bc = libmp.from_man_exp(v[0], v[1], p, "n")
        ref = Fraction(int(man)) * Fraction(2) ** int(exp) * (-1 if sign else 1)
        assert F(r) == ref


def test_rne_ties_even_handmade():
    # 2 bits: 5 = 101b -> tie between 4 and 6 -> 4 (even mantissa 10b); 7 = 111b -> 8; 3 -> 3
    assert F(X.rne((5, 0), 2)[0]) == 4
    assert F(X.rne((7, 0), 2)[0]) == 8
    assert F(X.rne((3, 0), 2)[0]) == 3
    assert F(X.rne((-5, 0), 2)[0]) == -4
    assert F(X.rne((11, 0), 3)[0]) == 12  # 1011b: tie -> 1100b
    assert F(X.rne((9, 0), 3)[0]) == 8  # 1001b: tie -> 1000b


def test_mag_from_upper_and_tight():
    rng = random.Random(3)
    for _ in range(2000):
        v = (rng.randint(0, 2**rng.randint(1, 120)), rng.randint(-500, 500))
        b, f = X.mag_from(v)
        if v[0] == 0:
            assert (b, f) == (0, 0)
            continue
        assert 2**29 <= b < 2**30
        up = Fraction(b) * Fraction(2) ** (f - 30)
        assert up >= F(v)
        assert up - F(v) < Fraction(2) ** (f - 30)  # within one unit of the 30-bit mantissa
    assert X.mag_from((1, 0)) == (2**29, 1)
    assert X.mag_from((2**30 - 1, 0)) == (2**30 - 1, 30)
    assert X.mag_from((2**31 - 1, 0)) == (2**29, 32)  # rounds up to 2^31 = 2^29 * 2^(32-30)


def test_mag_add_up_bounds_sum():
    rng = random.Random(4)
    for _ in range(1000):
        a = X.mag_from((rng.randint(1, 2**40), rng.randint(-100, 100)))
        b = X.mag_from((rng.randint(1, 2**40), rng.randint(-100, 100)))
        s = X.mag_add_up(a, b)
        exact = F(X.mag_value(a)) + F(X.mag_value(b))
        up = F(X.mag_value(s))
        assert up >= exact and up - exact < Fraction(2) ** (s[1] - 30)


def test_containment_and_ratio_handmade():
    S = (3, 0)
    R = (1, -2)  # 0.25
    assert X.contains((3, 0), X.mag_value(X.mag_from((1, -2))), S, R)
    assert not X.contains((3, 0), (1, -3), S, R)
    assert X.contains((13, -2), (1, 0), S, R)  # |3.25-3| + 0.25 = 0.5 <= 1
    assert X.accuracy_ratio((13, -2), S, (3, 0), 2) == pytest.approx(Fraction(1, 4) / Fraction(3, 4))


def test_special_values_are_rejected():
    raw = random_balls(0, 4, 1, 64, -3, 3)
    raw.flags[2] = FLAG_NAN
    with pytest.raises(X.Special):
        X.mid(raw, 2)
    raw2 = random_balls(0, 2, 1, 64, -3, 3)
    raw2.exp[1] = 1 << 60
    with pytest.raises(X.Special):
        X.mid(raw2, 1)


def test_result_exact_closed_forms():
    # N = 1: the midpoint is RNE_p(x*y)
    x = make_balls([Fraction(2**64 - 1, 2**64)], nlimbs=1)
    y = make_balls([Fraction(3)], nlimbs=1)
    m, r, S, _, _ = X.result_exact(X.real_dot_terms(x, [0], y, [0]), 2, 1)
    assert F(S) == Fraction(3 * (2**64 - 1), 2**64)
    assert F(m) == 3  # 2.99999... rounds to 3 at 2 bits
    # integer inputs, exact sum: radius zero
    x = make_balls([5, -7, 11])
    y = make_balls([3, 2, 1])
    m, r, S, _, R = X.result_exact(X.real_dot_terms(x, range(3), y, range(3)), 64, 1)
    assert F(m) == 15 - 14 + 11 and r == (0, 0)
    # x*1 - x*1 = 0 exactly
    x = make_balls([Fraction(-13, 1024), Fraction(-13, 1024)])
    y = make_balls([1, -1])
    m, r, S, _, _ = X.result_exact(X.real_dot_terms(x, range(2), y, range(2)), 64, 1)
    assert m[0] == 0 and r == (0, 0)


def test_ball_values_agree_with_oracle_decode():
    raw = random_balls(5, 50, 3, 150, -40, 40, rad_bits=100)
    for i in range(50):
        m, r = ball_values(raw, i)
        assert F(X.mid(raw, i)) == m and F(X.rad(raw, i)) == r


# ------------------------------------------------------------------ planted mistakes

def _fails(fn, *args):
    try:
        fn(*args)
    except (AssertionError, ValueError):  # a failed pin, or the decoder's own layout check
        return True
    return False


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the exact oracle makes at least one pin above fail, and every pin
    passes again once the slip is undone."""
    orig = {n: getattr(X, n) for n in ("limb_field", "dot_terms_exact", "complex_dot_terms",
                                       "rne", "mag_from")}

    # (a) limbs read most significant first
    def reversed_limbs(raw, i):
        v = 0
        for k in range(raw.nlimbs):
            v = (v << 64) | int(raw.limbs[k, i])
        return v
    monkeypatch.setattr(X, "limb_field", reversed_limbs)
    assert _fails(test_decode_handmade_multilimb)
    monkeypatch.setattr(X, "limb_field", orig["limb_field"])

    # (b) the last term of a dot dropped
    monkeypatch.setattr(X, "dot_terms_exact",
                        lambda terms, initial=None: orig["dot_terms_exact"](terms[:-1], initial))
    assert _fails(test_exact_dot_vs_fraction_bruteforce, 1)
    monkeypatch.setattr(X, "dot_terms_exact", orig["dot_terms_exact"])

    # (c) a wrong sign on b d in the real part of a complex product
    def re_plus_bd(x, xidx, y, yidx, sub=False):
        re, im = orig["complex_dot_terms"](x, xidx, y, yidx, sub)
        return [(a, c, bool(sub)) for a, c, _ in re], im
    monkeypatch.setattr(X, "complex_dot_terms", re_plus_bd)
    assert _fails(test_complex_terms_closed_form)
    monkeypatch.setattr(X, "complex_dot_terms", orig["complex_dot_terms"])

    # (d) ties rounded away from zero instead of to even
    def ties_away(v, p):
        num, e = v
        n = abs(num).bit_length()
        if n <= p:
            return orig["rne"](v, p)
        cut = n - p
        q, rem = divmod(abs(num), 1 << cut)
        if 2 * rem == (1 << cut):  # an exact tie
            r = ((q + 1) << cut) * (1 if num > 0 else -1)
            return (r, e), X.dy_abs(X.dy_add((r, e), X.dy_neg(v)))
        return orig["rne"](v, p)
    monkeypatch.setattr(X, "rne", ties_away)
    assert _fails(test_rne_ties_even_handmade)
    monkeypatch.setattr(X, "rne", orig["rne"])

    # (e) a radius magnitude rounded down instead of up
    def mag_down(v):
        b, f = orig["mag_from"](v)
        return (b - 1, f) if b > 2**29 else (b, f)
    monkeypatch.setattr(X, "mag_from", mag_down)
    assert _fails(test_mag_from_upper_and_tight)
    monkeypatch.setattr(X, "mag_from", orig["mag_from"])

    for fn, args in ((test_decode_handmade_multilimb, ()),
                     (test_exact_dot_vs_fraction_bruteforce, (1,)),
                     (test_complex_terms_closed_form, ()), (test_rne_ties_even_handmade, ()),
                     (test_mag_from_upper_and_tight, ())):
        assert not _fails(fn, *args)
