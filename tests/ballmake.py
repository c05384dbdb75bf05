"""Test-side construction of ball arrays from exact values (independent of the oracle's encoder)."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from synth import FLAG_SIGN, FLAG_ZERO, RawBalls


def frac_to_fields(v: Fraction, nlimbs: int):
    """Layout fields of a dyadic Fraction with at most 64*nlimbs significant bits."""
    if v == 0:
        return [0] * nlimbs, 0, FLAG_ZERO
    den = v.denominator
    assert den & (den - 1) == 0, "dyadic values only"
    a = abs(v)
    k = den.bit_length() - 1  # a = num / 2^k
    num = a.numerator
    L = num.bit_length()
    assert L <= 64 * nlimbs
    field = num << (64 * nlimbs - L)
    limbs = [(field >> (64 * j)) & ((1 << 64) - 1) for j in range(nlimbs)]
    e = L - k  # num/2^k in [2^(L-1-k), 2^(L-k))
    nsig = next(nlimbs - j for j in range(nlimbs) if limbs[j])
    return limbs, e, (FLAG_SIGN if v < 0 else 0) | (nsig << 8)


def rad_to_fields(r: Fraction):
    """Exact 30-bit radius fields of a dyadic Fraction with at most 30 significant bits."""
    if r == 0:
        return 0, 0
    m, e = math.frexp(float(r))
    assert Fraction(m) * Fraction(2) ** e == r
    man = int(Fraction(m) * (1 << 30))
    assert Fraction(man, 1 << 30) == Fraction(m)
    return man, e


def make_balls(mids, rads=None, nlimbs=1) -> RawBalls:
    n = len(mids)
    raw = RawBalls.zeros(n, nlimbs)
    for i, v in enumerate(mids):
        limbs, e, fl = frac_to_fields(Fraction(v), nlimbs)
        for j in range(nlimbs):
            raw.limbs[j, i] = np.uint64(limbs[j])
        raw.exp[i] = e
        raw.flags[i] = fl
        if rads is not None:
            man, re = rad_to_fields(Fraction(rads[i]))
            raw.rad_man[i] = man
            raw.rad_exp[i] = re
    return raw


def ball_values(raw, i):
    """Exact (mid, rad) Fractions of an entry, decoded here with floats/Fractions only."""
    fl = int(raw.flags[i])
    if fl & FLAG_ZERO:
        m = Fraction(0)
    else:
        field = 0
        for j in range(raw.nlimbs - 1, -1, -1):
            field = field * (1 << 64) + int(raw.limbs[j, i])
        m = Fraction(field) * Fraction(2) ** (int(raw.exp[i]) - 64 * raw.nlimbs)
        if fl & FLAG_SIGN:
            m = -m
    r = Fraction(int(raw.rad_man[i])) * Fraction(2) ** (int(raw.rad_exp[i]) - 30)
    return m, r
