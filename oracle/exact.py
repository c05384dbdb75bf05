"""Exact reference values for ball dot products and matrix products (test infrastructure only).

Numbers are exact dyadic rationals held as ``(num, e)`` pairs meaning ``num * 2**e`` with ``num`` a
Python integer.  Everything here is a direct transcription of a definition; nothing is blocked,
fused or reordered.

Definitions followed:

* Ball layout of a midpoint: ``m = (-1)^sign * 2^e * sum_k b_k 2^(64(k-n))`` (Section III-A, eq. 1),
  radius ``r = (b / 2^30) 2^f`` with ``p_rad = 30`` (Section III-A).
* Dot product of balls (Section II): the exact value ``S = sum m_i m'_i`` and the propagated radius
  ``R* = sum |m_i| r'_i + |m'_i| r_i + r_i r'_i``; an output ball ``[m +- r]`` is correct when
  ``|m - S| + R* <= r`` (containment), and accurate when ``|m - S| <= 2^-p * sum |m_i m'_i|``.
* The optional ``initial`` term and the ``sub`` flag of ``arb_dot`` (Section III): the result
  contains ``initial + (-1)^sub * sum x_i y_i``.
* A complex dot is two real dots over the real and imaginary parts (Section III-F); a matrix entry
  is the dot of a row and a column (Section IV).
"""
from __future__ import annotations

FLAG_SIGN = 1
FLAG_ZERO = 2
FLAG_INF = 4
FLAG_NAN = 8
FLAG_RAD_INF = 16
P_RAD = 30
EXP_LIMIT = 1 << 60  # exponents with |e| >= 2^60 are rejected as unsupported values


class Special(Exception):
    """An input holds a value the fixed-point path does not take (NaN, infinity, huge exponent)."""


# ----------------------------------------------------------------------------- dyadic helpers

def dy_add(a, b):
    if a[0] == 0:
        return b
    if b[0] == 0:
        return a
    e = min(a[1], b[1])
    return ((a[0] << (a[1] - e)) + (b[0] << (b[1] - e)), e)


def dy_neg(a):
    return (-a[0], a[1])


def dy_abs(a):
    return (abs(a[0]), a[1])


def dy_mul(a, b):
    return (a[0] * b[0], a[1] + b[1])


def dy_cmp(a, b) -> int:
    d = dy_add(a, dy_neg(b))[0]
    return (d > 0) - (d < 0)


def dy_sum(items):
    acc = (0, 0)
    for it in items:
        acc = dy_add(acc, it)
    return acc


def dy_to_fraction(a):
    from fractions import Fraction
    return Fraction(a[0]) * (Fraction(2) ** a[1])


# ----------------------------------------------------------------------------- layout decoding

def limb_field(raw, i) -> int:
    """The ``64*nlimbs``-bit unsigned integer formed by the limbs of entry ``i``."""
    v = 0
    for k in range(raw.nlimbs - 1, -1, -1):
        v = (v << 64) | int(raw.limbs[k, i])
    return v


def mid(raw, i):
    """Exact midpoint of entry ``i`` as a dyadic (Section III-A, eq. 1)."""
    fl = int(raw.flags[i])
    if fl & (FLAG_NAN | FLAG_INF):
        raise Special("non-finite midpoint")
    if fl & FLAG_ZERO:
        return (0, 0)
    e = int(raw.exp[i])
    if abs(e) >= EXP_LIMIT:
        raise Special("midpoint exponent out of range")
    v = limb_field(raw, i)
    if v >> (64 * raw.nlimbs - 1) != 1:
        raise ValueError("midpoint not normalised")
    return (-v if fl & FLAG_SIGN else v, e - 64 * raw.nlimbs)


def rad(raw, i):
    """Exact radius of entry ``i`` as a dyadic: ``rad_man * 2^(rad_exp - 30)``."""
    fl = int(raw.flags[i])
    if fl & FLAG_RAD_INF:
        raise Special("infinite radius")
    man = int(raw.rad_man[i])
    if man == 0:
        return (0, 0)
    f = int(raw.rad_exp[i])
    if abs(f) >= EXP_LIMIT:
        raise Special("radius exponent out of range")
    return (man, f - P_RAD)


def ball(raw, i):
    return mid(raw, i), rad(raw, i)


# ----------------------------------------------------------------------------- exact dot product

def dot_terms_exact(terms, initial=None):
    """Exact ``S``, ``sum |m_i m'_i|`` and ``R*`` of a dot product.

    ``terms`` holds ``((m, r), (m', r'), negate)`` triples of dyadics; ``initial`` is an optional
    ``(m, r)`` ball added with a plus sign (Section II, Section III)."""
    S = (0, 0)
    Sabs = (0, 0)
    R = (0, 0)
    for (m1, r1), (m2, r2), neg in terms:
        t = dy_mul(m1, m2)
        S = dy_add(S, dy_neg(t) if neg else t)
        Sabs = dy_add(Sabs, dy_abs(t))
        R = dy_add(R, dy_add(dy_add(dy_mul(dy_abs(m1), r2), dy_mul(dy_abs(m2), r1)),
                             dy_mul(r1, r2)))
    if initial is not None:
        m0, r0 = initial
        S = dy_add(S, m0)
        Sabs = dy_add(Sabs, dy_abs(m0))
        R = dy_add(R, r0)
    return S, Sabs, R


def real_dot_terms(x, xidx, y, yidx, sub=False):
    return [(ball(x, i), ball(y, j), bool(sub)) for i, j in zip(xidx, yidx)]


def complex_dot_terms(x, xidx, y, yidx, sub=False):
    """Real and imaginary term lists of a complex dot ``sum (a+bi)(c+di)``: the real part is
    ``sum ac - bd`` and the imaginary part ``sum ad + bc``, each a real dot of length 2N
    (Section III-F)."""
    xr, xi = x
    yr, yi = y
    re, im = [], []
    for i, j in zip(xidx, yidx):
        a, b, c, d = ball(xr, i), ball(xi, i), ball(yr, j), ball(yi, j)
        re.append((a, c, bool(sub)))
        re.append((b, d, not sub))
        im.append((a, d, bool(sub)))
        im.append((b, c, bool(sub)))
    return re, im


def matmul_entry_terms(A, B, K, N, i, j):
    """Terms of entry (i, j) of a real row-major product: row i of A times column j of B."""
    return real_dot_terms(A, [i * K + k for k in range(K)], B, [k * N + j for k in range(K)])


# ----------------------------------------------------------------------------- rounding

def rne(v, p):
    """Round the dyadic ``v`` to ``p`` significant bits, to nearest with ties to even.

    Returns ``(rounded_dyadic, error_dyadic)`` with ``error = |rounded - v|``."""
    num, e = v
    if num == 0:
        return (0, 0), (0, 0)
    s = -1 if num < 0 else 1
    a = abs(num)
    L = a.bit_length()
    if L <= p:
        return v, (0, 0)
    k = L - p
    q = a >> k
    rem = a - (q << k)
    half = 1 << (k - 1)
    if rem > half or (rem == half and (q & 1)):
        q += 1
        err = (1 << k) - rem
    else:
        err = rem
    return (s * (q << k), e), (err, e)


# ----------------------------------------------------------------------------- 30-bit radii

def mag_from(v):
    """Smallest 30-bit radius ``b * 2^(f-30)``, ``2^29 <= b < 2^30``, that is ``>= v >= 0``.

    Returns ``(b, f)``; zero is ``(0, 0)``.  (Upward rounding of the radius, Section III-A/E.)"""
    num, e = v
    if num < 0:
        raise ValueError("negative radius")
    if num == 0:
        return (0, 0)
    L = num.bit_length()
    if L <= P_RAD:
        return (num << (P_RAD - L), e + L)
    b = num >> (L - P_RAD)
    if b << (L - P_RAD) != num:
        b += 1
    f = e + L
    if b == 1 << P_RAD:
        b >>= 1
        f += 1
    return (b, f)


def mag_value(m):
    b, f = m
    return (b, f - P_RAD) if b else (0, 0)


def mag_add_up(a, b):
    """Upper bound of a sum of two 30-bit radii, rounded up to 30 bits (exact sum, one rounding)."""
    return mag_from(dy_add(mag_value(a), mag_value(b)))


# ----------------------------------------------------------------------------- encoding

def encode_mid(v, nlimbs):
    """Layout fields ``(limbs list little-endian, exp, flags)`` of the dyadic ``v``; ``v`` must fit
    in ``64*nlimbs`` significant bits."""
    num, e = v
    if num == 0:
        return [0] * nlimbs, 0, FLAG_ZERO
    a = abs(num)
    tz = (a & -a).bit_length() - 1
    a >>= tz
    e += tz
    L = a.bit_length()
    if L > 64 * nlimbs:
        raise ValueError("too many bits for nlimbs")
    field = a << (64 * nlimbs - L)
    limbs = [(field >> (64 * k)) & ((1 << 64) - 1) for k in range(nlimbs)]
    nsig = 0
    for k in range(nlimbs):
        if limbs[k] != 0:
            nsig = nlimbs - k
            break
    flags = (FLAG_SIGN if num < 0 else 0) | (nsig << 8)
    return limbs, e + L, flags


def result_exact(terms, prec, nlimbs_out, initial=None):
    """The exactly rounded ball: midpoint ``RNE_p(S)`` and radius ``mag_from(|RNE_p(S) - S| + R*)``.

    This is the best ball a p-bit midpoint with a 30-bit upward radius can give."""
    S, Sabs, R = dot_terms_exact(terms, initial)
    m, err = rne(S, prec)
    return m, mag_from(dy_add(err, R)), S, Sabs, R


# ----------------------------------------------------------------------------- checks

def decode_output(raw, i):
    """(midpoint, radius) of an output entry, or None for the unsupported-value marker."""
    fl = int(raw.flags[i])
    if fl & (FLAG_NAN | FLAG_INF | FLAG_RAD_INF):
        return None
    return mid(raw, i), rad(raw, i)


def contains(m, r, S, R) -> bool:
    """Containment: every point of the input balls maps into ``[m +- r]``, i.e.
    ``|m - S| + R* <= r`` (Section II)."""
    lhs = dy_add(dy_abs(dy_add(m, dy_neg(S))), R)
    return dy_cmp(lhs, r) <= 0


def accuracy_ratio(m, S, Sabs, p) -> float:
    """``|m - S| / (2^-p * sum |m_i m'_i|)`` as a float (0 when both are zero)."""
    from fractions import Fraction
    d = dy_to_fraction(dy_abs(dy_add(m, dy_neg(S))))
    den = dy_to_fraction(Sabs) / (Fraction(2) ** p)
    if den == 0:
        return 0.0 if d == 0 else float("inf")
    return float(d / den)
