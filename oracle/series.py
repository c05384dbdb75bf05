"""The power series exponential of Section V, restated on exact rationals (test infrastructure only).

Section V gives the dot-product recurrence that the basecase of the series exponential uses:

    exp(a_1 x + a_2 x^2 + ...) = b_0 + b_1 x + b_2 x^2 + ...,   b_0 = 1,
    b_k = (sum_{j=1}^k (j a_j) b_{k-j}) / k.

``exp_series`` is that recurrence on ``fractions.Fraction`` values (exact).  ``exp_series_radius``
is the radius that exact ball arithmetic propagates through the same recurrence when each a_j is
known only to within rho_j: with |a_j| and |b_{k-j}| bounds and the radii r_{k-j} of earlier
coefficients,

    r_0 = 0,   r_k = (sum_{j=1}^k j (|a_j| r_{k-j} + rho_j |b_{k-j}| + rho_j r_{k-j})) / k,

an upper bound of |b_k(a') - b_k(a)| for every a' with |a'_j - a_j| <= rho_j (the product rule of
Section II term by term).  An output ball [m +- r] of coefficient k is correct when
|m - b_k| + r_k <= r.
"""
from __future__ import annotations

from fractions import Fraction


def exp_series(a, n):
    """Coefficients b_0 .. b_{n-1} of exp(a_1 x + a_2 x^2 + ...); ``a[0]`` is ignored."""
    b = [Fraction(0)] * n
    if n == 0:
        return b
    b[0] = Fraction(1)
    for k in range(1, n):
        s = Fraction(0)
        for j in range(1, k + 1):
            aj = a[j] if j < len(a) else Fraction(0)
            s += (j * aj) * b[k - j]
        b[k] = s / k
    return b


def exp_series_radius(a, rho, n):
    """Propagated radii r_0 .. r_{n-1} of the coefficients for inputs a_j +- rho_j."""
    b = exp_series(a, n)
    r = [Fraction(0)] * n
    for k in range(1, n):
        s = Fraction(0)
        for j in range(1, k + 1):
            aj = abs(a[j]) if j < len(a) else Fraction(0)
            pj = rho[j] if j < len(rho) else Fraction(0)
            s += j * (aj * r[k - j] + pj * abs(b[k - j]) + pj * r[k - j])
        r[k] = s / k
    return b, r
