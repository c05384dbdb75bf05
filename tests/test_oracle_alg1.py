"""Pins for the Algorithm 1 restatement (``oracle.alg1``): the hand-traced worked example, the
paper's invariants checked against the exact oracle (itself pinned in test_oracle_exact.py), closed
forms, and planted mistakes that the pins must catch."""
from __future__ import annotations

import json
import os
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import alg1
from oracle import exact as X
from synth import RawBalls, random_balls
from tests.ballmake import make_balls

GOLD = os.path.join(os.path.dirname(__file__), "golden", "alg1_worked_example.json")


def F(d):
    return X.dy_to_fraction(d)


def out_mid_rad(res, nlimbs):
    raw = RawBalls.zeros(1, nlimbs)
    for k in range(nlimbs):
        raw.limbs[k, 0] = np.uint64(res["limbs"][k])
    raw.exp[0] = res["exp"]
    raw.flags[0] = res["flags"]
    raw.rad_man[0] = res["rad_man"]
    raw.rad_exp[0] = res["rad_exp"]
    return X.mid(raw, 0), X.rad(raw, 0)


def worked_example(rx0=0):
    x = make_balls([1, Fraction(1, 2**200), Fraction(3, 2**70)], [rx0, 0, 0])
    y = make_balls([1, 1, 1])
    return alg1.dot(alg1.real_terms(x, range(3), y, range(3)), 2, 1)


def check_golden(dotfun=None):
    g = json.load(open(GOLD))
    r = worked_example() if dotfun is None else dotfun()
    e = g["expect_no_radius"]
    ok = (r["err"] == e["err"] and r["n_s"] == e["n_s"] and r["e_s"] == e["e_s"]
          and F(out_mid_rad(r, 1)[0]) == 1 and (r["rad_man"], r["rad_exp"]) == (e["rad_man"],
                                                                                   e["rad_exp"]))
    r2 = worked_example(Fraction(2**30 - 1, 2**40))
    w = g["with_radius_on_x0"]
    ok = ok and (r2["srad"], r2["e_rad"], r2["rad_man"], r2["rad_exp"]) == (
        w["srad"], w["e_rad"], w["rad_man"], w["rad_exp"])
    return ok


def test_worked_example_matches_hand_trace():
    assert check_golden()


def _case(seed, n, prec, nl, exp_spread, rad_bits, rad_zero, zero_frac=0.0, sub=False,
          with_init=False):
    rng = np.random.default_rng(seed)
    mb = rng.integers(1, 64 * nl + 1, size=n)
    x = random_balls(rng, n, nl, mb, -exp_spread, exp_spread, rad_bits=rad_bits,
                     rad_zero_frac=rad_zero, zero_frac=zero_frac)
    y = random_balls(rng, n, nl, mb[::-1].copy(), -exp_spread, exp_spread, rad_bits=rad_bits,
                     rad_zero_frac=rad_zero, zero_frac=zero_frac)
    init = random_balls(rng, 1, nl, 64 * nl, -exp_spread, exp_spread, rad_bits=rad_bits) \
        if with_init else None
    return x, y, init


CASES = [
    # (n, prec, nlimbs, exponent spread, radius bits, zero-radius fraction, zero fraction, sub, init)
    (1, 2, 1, 4, None, 0, 0, False, False),
    (5, 64, 1, 10, None, 0, 0, False, False),
    (7, 53, 2, 200, 40, 0.5, 0.2, True, True),
    (32, 128, 2, 8, None, 0, 0, False, False),
    (40, 128, 3, 300, 120, 0.5, 0.1, False, True),
    (17, 192, 3, 30, 190, 0.5, 0, True, False),
    (64, 256, 4, 20, 250, 0, 0, False, False),
    (9, 1024, 16, 3000, 1000, 0.3, 0.1, True, True),
    (33, 65, 2, 64, 60, 0.0, 0.3, False, False),
    (3, 3, 1, 1, 2, 0.0, 0.0, False, False),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("seed", range(6))
def test_invariants_against_exact(case, seed):
    n, prec, nl, spread, rb, rz, zf, sub, wi = CASES[case]
    x, y, init = _case(1000 * case + seed, n, prec, nl, spread, rb, rz, zf, sub, wi)
    terms = alg1.real_terms(x, range(n), y, range(n), sub)
    ient = alg1.entry(init, 0) if init is not None else None
    res = alg1.dot(terms, prec, (prec + 63) // 64, ient)
    assert res["status"] == 0
    xt = X.real_dot_terms(x, range(n), y, range(n), sub)
    S, Sabs, R = X.dot_terms_exact(xt, X.ball(init, 0) if init is not None else None)
    m, r = out_mid_rad(res, (prec + 63) // 64)
    # 1. containment (Section II)
    assert X.contains(m, r, S, R)
    # 2. rigorous accuracy: |m - S| <= half an ulp of m at p bits + err ulps of the accumulator
    if res["n_s"]:
        half_ulp = Fraction(2) ** (res["exp"] - prec - 1) if m[0] else 0
        trunc = res["err"] * Fraction(2) ** (res["e_s"] - 64 * res["n_s"])
        assert abs(F(m) - F(S)) <= half_ulp + trunc
        # the truncation term is far below 2^-p relative (padding guard bits)
        if Sabs[0]:
            assert trunc <= F(Sabs) * Fraction(2) ** (-prec - 4) * (res["err"] + 1)
    # 3. exactness (Section II): exact inputs + nothing truncated + S fits in p bits
    if res["err"] == 0 and R[0] == 0:
        mS, _ = X.rne(S, prec)
        if mS == S or F(mS) == F(S):
            assert F(m) == F(S) and r == (0, 0)


def test_midpoint_error_bound_on_random_signs():
    """|m - S| <= 2^-p sum |x y| (the dot's accuracy guarantee, Section III) on 40 random dots
    with mixed signs."""
    worst = 0.0
    for seed in range(40):
        x, y, _ = _case(seed, 50, 128, 2, 30, None, 0)
        res = alg1.dot(alg1.real_terms(x, range(50), y, range(50)), 128, 2)
        S, Sabs, R = X.dot_terms_exact(X.real_dot_terms(x, range(50), y, range(50)))
        m, _ = out_mid_rad(res, 2)
        worst = max(worst, X.accuracy_ratio(m, S, Sabs, 128))
    assert worst <= 1.0


def test_integer_inputs_give_exact_zero_radius():
    xs = [5, -7, 11, 2**40, -(2**40)]
    ys = [3, 2, 1, 9, 9]
    x, y = make_balls(xs), make_balls(ys)
    res = alg1.dot(alg1.real_terms(x, range(5), y, range(5)), 64, 1)
    m, r = out_mid_rad(res, 1)
    assert F(m) == 15 - 14 + 11 and r == (0, 0) and res["err"] == 0


def test_cancellation_gives_exact_zero():
    x = make_balls([Fraction(-13, 1024), Fraction(-13, 1024)])
    y = make_balls([1, -1])
    res = alg1.dot(alg1.real_terms(x, range(2), y, range(2)), 64, 1)
    assert res["flags"] == X.FLAG_ZERO and res["rad_man"] == 0


def test_single_term_is_rounded_product():
    rng = random.Random(11)
    for _ in range(200):
        p = rng.choice([2, 3, 53, 64, 100, 128])
        a = Fraction(rng.randint(1, 2**64 - 1), 2**rng.randint(0, 80)) * rng.choice([-1, 1])
        b = Fraction(rng.randint(1, 2**64 - 1), 2**rng.randint(0, 80)) * rng.choice([-1, 1])
        x, y = make_balls([a], nlimbs=1), make_balls([b], nlimbs=1)
        res = alg1.dot(alg1.real_terms(x, [0], y, [0]), p, (p + 63) // 64)
        m, _ = out_mid_rad(res, (p + 63) // 64)
        prod = a * b
        num, den = prod.numerator, prod.denominator
        e = -(den.bit_length() - 1)
        ref, _ = X.rne((num, e), p)
        assert F(m) == F(ref)


def test_initial_and_sub():
    x = make_balls([Fraction(3, 4), Fraction(1, 8)])
    y = make_balls([2, -4])
    init = make_balls([Fraction(5)])
    res = alg1.dot(alg1.real_terms(x, range(2), y, range(2), sub=True), 64, 1, alg1.entry(init, 0))
    m, _ = out_mid_rad(res, 1)
    assert F(m) == 5 - (Fraction(3, 2) - Fraction(1, 2))


def test_special_values_flagged():
    x = random_balls(1, 3, 1, 64, -3, 3)
    y = random_balls(2, 3, 1, 64, -3, 3)
    x.flags[1] = X.FLAG_INF
    res = alg1.dot_raw(x, range(3), y, range(3), 64, 1)
    assert res["status"] == 2 and res["flags"] & X.FLAG_NAN


def test_negative_strides_same_value():
    x, y, _ = _case(3, 12, 128, 2, 10, 100, 0.5)
    fwd = alg1.dot_raw(x, range(12), y, range(12), 128, 2)
    rev = alg1.dot_raw(x, range(11, -1, -1), y, range(11, -1, -1), 128, 2)
    assert fwd == rev  # order independence of the integer accumulation


# ------------------------------------------------------------------ planted mistakes

def _planted(monkeypatch, name, fn):
    monkeypatch.setattr(alg1, name, fn)


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the restatement makes at least one pin above fail."""
    orig_upper = alg1.mag_upper_of_mid
    orig_bc = alg1.bc

    # (a) radius upper bound without the +1
    monkeypatch.setattr(alg1, "mag_upper_of_mid", lambda x: (x.top[0] >> 34, x.e))
    assert not check_golden()
    monkeypatch.setattr(alg1, "mag_upper_of_mid", orig_upper)
    assert check_golden()

    # (b) wrong binary length in the setup (one too many) changes n_s / e_s
    monkeypatch.setattr(alg1, "bc", lambda v: v.bit_length() + 1)
    assert not check_golden()
    monkeypatch.setattr(alg1, "bc", orig_bc)

    # (c) a sign slip in the midpoint accumulation breaks containment
    orig_dot = alg1._dot

    def flipped(terms, prec, nl, init):
        return orig_dot([(a, b, not n) for a, b, n in terms], prec, nl, init)

    x, y, _ = _case(5, 6, 64, 1, 3, None, 0)
    S, Sabs, R = X.dot_terms_exact(X.real_dot_terms(x, range(6), y, range(6)))
    res = flipped(alg1.real_terms(x, range(6), y, range(6)), 64, 1, None)
    m, r = out_mid_rad(res, 1)
    assert not X.contains(m, r, S, R)

    # (d) a dropped term breaks containment
    res = alg1.dot(alg1.real_terms(x, range(5), y, range(5)), 64, 1)
    m, r = out_mid_rad(res, 1)
    assert not X.contains(m, r, S, R)


# ---- the "optimize p" step of Section III-C, asked for with reduce_prec

@pytest.mark.parametrize("seed", range(8))
def test_reduced_precision_keeps_a_result_that_fits_its_window(seed):
    """The paper: when all terms fit in a window smaller than p bits, reducing the precision does
    not change the result.  One-limb mantissas with exponents within +-6 at p = 256 fit (the exact
    sum has fewer than 190 bits), so the reduced run must give the same exact ball."""
    x, y, _ = _case(7000 + seed, 24, 256, 1, 6, None, 0)
    terms = alg1.real_terms(x, range(24), y, range(24))
    full = alg1.dot(terms, 256, 4)
    red = alg1.dot(terms, 256, 4, reduce_prec=True)
    assert red["prec"] < 256  # the window rule fired
    assert (red["limbs"], red["exp"], red["flags"]) == (full["limbs"], full["exp"], full["flags"])
    assert (red["rad_man"], full["rad_man"]) == (0, 0)
    S, _, _ = X.dot_terms_exact(X.real_dot_terms(x, range(24), y, range(24)))
    assert F(out_mid_rad(red, 4)[0]) == F(S)


@pytest.mark.parametrize("seed", range(8))
def test_reduced_precision_with_wide_radii_still_contains_the_exact_sum(seed):
    """Radii near 2^-40 relative: the radius rule lowers p to about 70 bits.  The ball must still
    contain the exact dot product, and its midpoint has at most the reduced number of bits."""
    x, y, init = _case(7100 + seed, 30, 256, 4, 20, 40, 0.3, with_init=True)
    terms = alg1.real_terms(x, range(30), y, range(30))
    res = alg1.dot(terms, 256, 4, alg1.entry(init, 0), reduce_prec=True)
    assert res["status"] == 0 and 2 <= res["prec"] < 128
    S, Sabs, R = X.dot_terms_exact(X.real_dot_terms(x, range(30), y, range(30)), X.ball(init, 0))
    m, r = out_mid_rad(res, 4)
    assert X.contains(m, r, S, R)
    mf = F(m)
    if mf:
        num = abs(mf.numerator) // (abs(mf.numerator) & -abs(mf.numerator))  # odd part
        assert num.bit_length() <= res["prec"]


def test_reduced_precision_of_a_zero_midpoint_is_two_bits():
    """Only radii: e_max is MIN, so p becomes 2 and the result is [0 +- r]."""
    x = make_balls([0, 0], [Fraction(1, 2**10), 0])
    y = make_balls([1, 1], [0, Fraction(1, 2**5)])
    res = alg1.dot(alg1.real_terms(x, range(2), y, range(2)), 128, 2, reduce_prec=True)
    assert res["prec"] == 2
    m, r = out_mid_rad(res, 2)
    assert F(m) == 0 and F(r) > 0


# ---- complex dots (Section III-F): two real dots of length 2N, ac - bd and ad + bc

def _complex_case(seed, n, prec, nl, spread, rad_bits):
    rng = np.random.default_rng(seed)
    mk = lambda: random_balls(rng, n, nl, 64 * nl, -spread, spread, rad_bits=rad_bits,  # noqa
                              rad_zero_frac=0.5, zero_frac=0.1)
    return (mk(), mk()), (mk(), mk())


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("sub,with_init", [(False, False), (True, True)])
def test_complex_dot_against_exact(seed, sub, with_init):
    n, prec, nl = 9, 128, 2
    x, y = _complex_case(50 + seed, n, prec, nl, 40, 120)
    init = None
    if with_init:
        rng = np.random.default_rng(seed)
        init = ((random_balls(rng, 1, nl, 128, -5, 5, rad_bits=100),
                 random_balls(rng, 1, nl, 128, -5, 5, rad_bits=100)), 0)
    re, im = alg1.complex_dot_raw(x, range(n), y, range(n), prec, nl, sub=sub, initial=init)
    xre, xim = X.complex_dot_terms(x, range(n), y, range(n), sub=sub)
    for res, terms, q in ((re, xre, 0), (im, xim, 1)):
        ib = X.ball(init[0][q], 0) if init else None
        S, Sabs, R = X.dot_terms_exact(terms, ib)
        m, r = out_mid_rad(res, nl)
        assert X.contains(m, r, S, R)
        assert X.accuracy_ratio(m, S, Sabs, prec) <= 1.0


def test_complex_single_term_closed_form():
    """(3/4 - 5/8 i)(7/2 + 1/16 i) = (21/8 + 5/128) + (3/64 - 35/16) i, exact at p = 64."""
    x = (make_balls([Fraction(3, 4)]), make_balls([Fraction(-5, 8)]))
    y = (make_balls([Fraction(7, 2)]), make_balls([Fraction(1, 16)]))
    re, im = alg1.complex_dot_raw(x, [0], y, [0], 64, 1)
    assert F(out_mid_rad(re, 1)[0]) == Fraction(21, 8) + Fraction(5, 128)
    assert F(out_mid_rad(im, 1)[0]) == Fraction(3, 64) - Fraction(35, 16)
    assert out_mid_rad(re, 1)[1] == (0, 0) and out_mid_rad(im, 1)[1] == (0, 0)


def test_planted_complex_sign_slip_is_caught(monkeypatch):
    """b d added instead of subtracted in the real part: containment fails."""
    orig = alg1.complex_terms

    def plus_bd(x, xidx, y, yidx, sub=False):
        re, im = orig(x, xidx, y, yidx, sub)
        return [(a, c, bool(sub)) for a, c, _ in re], im
    monkeypatch.setattr(alg1, "complex_terms", plus_bd)
    x, y = _complex_case(77, 6, 128, 2, 10, None)
    re, _ = alg1.complex_dot_raw(x, range(6), y, range(6), 128, 2)
    xre, _ = X.complex_dot_terms(x, range(6), y, range(6))
    S, Sabs, R = X.dot_terms_exact(xre)
    m, r = out_mid_rad(re, 2)
    assert not X.contains(m, r, S, R)
