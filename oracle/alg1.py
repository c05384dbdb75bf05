"""Algorithm 1 of the paper (Section III), restated on Python integers (test infrastructure only).

This is the step-by-step reference for the warp-per-dot kernel: the same setup quantities, the same
per-term truncation decisions and the same final rounding, so that its output must agree bit for
bit.  The accumulation is integer arithmetic modulo ``2^(64 n_s)`` and every truncation decision
depends on one term only, so the order in which terms are added does not change the result.

Steps (Section III-B..E):

* Setup (Section III-C): reject non-finite values and exponents with ``|e| >= 2^60`` (where the
  paper leaves the fixed-point path for a fallback); count the terms with two nonzero midpoints,
  ``e_max = max(e + e')``, ``e_rad`` = largest exponent of a nonzero radius product; return
  ``[0 +- 0]`` when there is nothing; ``padding = 4 + bc(N)``, ``extend = bc(N_nonzero) + 1``,
  ``n_s = max(2, ceil((p + extend + padding) / 64))``, ``e_s = e_max + extend``.
* Evaluation (Section III-D): ``shift = e_s - (e + e')``; a term with ``shift >= 64 n_s`` only adds
  one ulp to ``err``; otherwise at most ``n'' = ceil(p_t / 64) + 1`` leading limbs of each factor are
  read (one ulp if a factor is cut), their exact product is aligned to the accumulator and added or
  subtracted in two's complement; nonzero bits falling below the accumulator add one ulp.
* Radius (Section III-E): each midpoint becomes the 30-bit upper bound "top 30 bits of the top limb,
  plus one"; each nonzero product adds ``floor(ab / 2^(30 + e_rad - e)) + 1`` (or 1) to ``srad``.
* Finalisation (Algorithm 1's last phase): negate if the top bit is set, round to ``p`` bits, and bound
  ``eps_round + err * 2^(e_s - 64 n_s) + srad * 2^(e_rad - 30)`` by a 30-bit radius.

Readings where the paper leaves a choice (each also used by the kernel):

* Rounding to p bits is round-to-nearest, ties to even.
* The precision reduction of Section III-C ("optimize p") is applied only when asked
  (``reduce_prec``); by default p stays as given.
* ``initial`` is the extra term ``initial * 1`` with the exact ball ``[1 +- 0]`` (Section III-B:
  "extending the dot product to length N + 1"); ``N`` in ``padding`` counts it.
* The radius is formed as: the integer ``eps_round + err`` (both in accumulator ulps) rounded up to
  30 bits, ``srad`` rounded up to 30 bits, then their sum rounded up to 30 bits.
* Unsupported values make the output ``[NaN +- inf]`` and raise a status flag.
"""
from __future__ import annotations

from .exact import (EXP_LIMIT, FLAG_INF, FLAG_NAN, FLAG_RAD_INF, FLAG_SIGN, FLAG_ZERO, P_RAD,
                    Special, encode_mid, mag_add_up, mag_from, rne)

BETA = 64
MASK64 = (1 << 64) - 1


class Entry:
    """One ball as Algorithm 1 sees it: sign, exponent, limb count and the significant limbs."""

    __slots__ = ("zero", "sign", "e", "n", "top", "rman", "rexp")

    def __init__(self, zero, sign, e, n, top, rman, rexp):
        self.zero, self.sign, self.e, self.n, self.top = zero, sign, e, n, top
        self.rman, self.rexp = rman, rexp

    def leading(self, count):
        """Integer formed by the ``count`` most significant limbs (count <= n)."""
        v = 0
        for k in range(count):
            v = (v << BETA) | self.top[k]
        return v


ONE = Entry(False, 0, 1, 1, [1 << 63], 0, 0)


def entry(raw, i) -> Entry:
    fl = int(raw.flags[i])
    if fl & (FLAG_NAN | FLAG_INF | FLAG_RAD_INF):
        raise Special("non-finite value")
    rman = int(raw.rad_man[i])
    rexp = int(raw.rad_exp[i])
    if rman and abs(rexp) >= EXP_LIMIT:
        raise Special("radius exponent out of range")
    if fl & FLAG_ZERO:
        return Entry(True, 0, 0, 0, [], rman, rexp)
    e = int(raw.exp[i])
    if abs(e) >= EXP_LIMIT:
        raise Special("exponent out of range")
    n = (fl >> 8) & 0xFF
    nl = raw.nlimbs
    top = [int(raw.limbs[nl - 1 - k, i]) for k in range(n)]
    return Entry(False, fl & FLAG_SIGN, e, n, top, rman, rexp)


def bc(v: int) -> int:
    """Binary length ``ceil(log2(v + 1))``."""
    return v.bit_length()


def mag_upper_of_mid(x: Entry):
    """30-bit upper bound of |m|: the top 30 bits of the top limb, plus one (weakly normalised)."""
    return (x.top[0] >> (BETA - P_RAD)) + 1, x.e


def dot(terms, prec, nlimbs_out, initial=None, reduce_prec=False):
    """Algorithm 1 on ``terms`` = list of ``(Entry, Entry, negate)``.

    Returns a dict with the output layout fields (``limbs``, ``exp``, ``flags``, ``rad_man``,
    ``rad_exp``), ``status`` (0 or 2 for an unsupported value) and the internal quantities.  With
    ``reduce_prec``, the "optimize p" step of Section III-C lowers the working and output precision."""
    try:
        return _dot(terms, prec, nlimbs_out, initial, reduce_prec)
    except Special:
        return dict(limbs=[0] * nlimbs_out, exp=0, flags=FLAG_NAN | FLAG_RAD_INF, rad_man=0,
                    rad_exp=0, status=2)


def _dot(terms, prec, nlimbs_out, initial, reduce_prec=False):
    if prec < 2:
        raise ValueError("p >= 2")
    allt = list(terms)
    if initial is not None:
        allt.append((initial, ONE, False))
    N = len(allt)

    # ---- setup pass
    n_nonzero = 0
    e_max = None
    e_rad = None
    e_min = None  # lowest possible bit of a product, tracked when p > 2 beta (Section III-C)
    for x, y, _neg in allt:
        if not x.zero and not y.zero:
            n_nonzero += 1
            t = x.e + y.e
            e_max = t if e_max is None else max(e_max, t)
            if prec > 2 * BETA:
                lo = t - BETA * (x.n + y.n)
                e_min = lo if e_min is None else min(e_min, lo)
        for ee in _radius_exponents(x, y):
            e_rad = ee if e_rad is None else max(e_rad, ee)
    if e_max is None and e_rad is None:
        return dict(limbs=[0] * nlimbs_out, exp=0, flags=FLAG_ZERO, rad_man=0, rad_exp=0,
                    status=0, n_s=0, e_s=0, err=0, srad=0, e_rad=None)
    if reduce_prec:  # "optimize p": a radius above the arithmetic error, or a narrow window of terms
        if e_max is None:
            prec = 2
        else:
            if e_rad is not None:
                prec = min(prec, e_max - e_rad + P_RAD)
            if e_min is not None:
                prec = min(prec, e_max - e_min + P_RAD)
            prec = max(prec, 2)
    padding = 4 + bc(N)
    extend = bc(n_nonzero) + 1
    n_s = max(2, -(-(prec + extend + padding) // BETA))
    e_s = (e_max + extend) if e_max is not None else 0
    width = BETA * n_s
    modulus = 1 << width

    # ---- evaluation
    s = 0
    err = 0
    srad = 0
    for x, y, neg in allt:
        if not x.zero and not y.zero:
            shift = e_s - (x.e + y.e)
            if shift >= width:
                err += 1
            else:
                p_t = width - shift
                n2 = -(-p_t // BETA) + 1
                if x.n > n2 or y.n > n2:
                    err += 1
                nx, ny = min(x.n, n2), min(y.n, n2)
                t = x.leading(nx) * y.leading(ny)
                q = width - shift - BETA * (nx + ny)
                if q >= 0:
                    a = t << q
                else:
                    a = t >> (-q)
                    if t & ((1 << (-q)) - 1):
                        err += 1
                negative = (x.sign ^ y.sign ^ (1 if neg else 0)) == 1
                s = (s - a) % modulus if negative else (s + a) % modulus
        for a_man, b_man, ee in _radius_products(x, y):
            d = e_rad - ee
            if d < P_RAD:
                srad += ((a_man * b_man) >> (P_RAD + d)) + 1
            else:
                srad += 1

    # ---- finalisation
    sign = 0
    if s >> (width - 1):
        s = modulus - s
        sign = 1
    ulp_e = e_s - width
    m, eps = rne(((-s if sign else s), ulp_e), prec)
    eps_int = eps[0] << (eps[1] - ulp_e) if eps[0] else 0
    r_mid = mag_from((eps_int + err, ulp_e))
    r_rad = mag_from((srad, e_rad - P_RAD)) if e_rad is not None else (0, 0)
    rman, rexp = mag_add_up(r_mid, r_rad)
    limbs, exp, flags = encode_mid(m, nlimbs_out)
    return dict(limbs=limbs, exp=exp, flags=flags, rad_man=rman, rad_exp=rexp, status=0,
                n_s=n_s, e_s=e_s, err=err, srad=srad, e_rad=e_rad, sign=sign, prec=prec)


def _radius_exponents(x, y):
    out = []
    if not x.zero and y.rman:
        out.append(x.e + y.rexp)
    if not y.zero and x.rman:
        out.append(y.e + x.rexp)
    if x.rman and y.rman:
        out.append(x.rexp + y.rexp)
    return out


def _radius_products(x, y):
    out = []
    if not x.zero and y.rman:
        a, ea = mag_upper_of_mid(x)
        out.append((a, y.rman, ea + y.rexp))
    if not y.zero and x.rman:
        a, ea = mag_upper_of_mid(y)
        out.append((a, x.rman, ea + x.rexp))
    if x.rman and y.rman:
        out.append((x.rman, y.rman, x.rexp + y.rexp))
    return out


# ----------------------------------------------------------------------------- convenience

def real_terms(xraw, xidx, yraw, yidx, sub=False):
    return [(entry(xraw, i), entry(yraw, j), bool(sub)) for i, j in zip(xidx, yidx)]


def complex_terms(x, xidx, y, yidx, sub=False):
    """Real-part and imaginary-part term lists of a complex dot (Section III-F): ``ac - bd`` and
    ``ad + bc``, each a real dot of length 2N."""
    xr, xi = x
    yr, yi = y
    re, im = [], []
    for i, j in zip(xidx, yidx):
        a, b, c, d = entry(xr, i), entry(xi, i), entry(yr, j), entry(yi, j)
        re.append((a, c, bool(sub)))
        re.append((b, d, not sub))
        im.append((a, d, bool(sub)))
        im.append((b, c, bool(sub)))
    return re, im


SPECIAL_OUTPUT = dict(limbs=None, exp=0, flags=FLAG_NAN | FLAG_RAD_INF, rad_man=0, rad_exp=0,
                      status=2)


def dot_raw(xraw, xidx, yraw, yidx, prec, nlimbs_out, sub=False, initial=None,
            reduce_prec=False):
    """Algorithm 1 on entries of raw ball arrays; ``initial`` is ``(raw, index)`` or None."""
    try:
        terms = real_terms(xraw, xidx, yraw, yidx, sub)
        init = entry(*initial) if initial is not None else None
    except Special:
        return dict(SPECIAL_OUTPUT, limbs=[0] * nlimbs_out)
    return dot(terms, prec, nlimbs_out, init, reduce_prec)


def complex_dot_raw(x, xidx, y, yidx, prec, nlimbs_out, sub=False, initial=None):
    """Complex dot: ``(re_result, im_result)``; ``initial`` is ``((re_raw, im_raw), index)``."""
    try:
        re, im = complex_terms(x, xidx, y, yidx, sub)
        ire = entry(initial[0][0], initial[1]) if initial is not None else None
        iim = entry(initial[0][1], initial[1]) if initial is not None else None
    except Special:
        sp = dict(SPECIAL_OUTPUT, limbs=[0] * nlimbs_out)
        return sp, dict(sp)
    return dot(re, prec, nlimbs_out, ire), dot(im, prec, nlimbs_out, iim)


def matmul_entry(A, B, K, N, i, j, prec, nlimbs_out):
    """Entry (i, j) of a real row-major product by Algorithm 1 (the classical algorithm)."""
    return dot_raw(A, [i * K + k for k in range(K)], B, [k * N + j for k in range(K)], prec,
                   nlimbs_out)
