"""Algorithm 2 of the paper (Section IV-A), restated on Python integers (test infrastructure only).

Steps, in the paper's order:

* ``h = 1.25 * min(p, max(p_A, p_B)) + 192`` where ``p_M`` is the least precision that holds every
  entry of ``M`` exactly (Algorithm 2's height bound).
* Greedy extraction (Section IV-A): starting at the first unused inner index, append indices while
  every row of ``A_s`` and every column of ``B_s`` still scales to integers of height below ``2^h``.
* A block of fewer than 30 indices is widened to ``min(30, |S|)`` indices and done with dot products
  (the basecase); otherwise ``T = (E_s A_s)(B_s F_s)`` over the integers, where ``E_s`` and ``F_s``
  hold the optimal (minimal-height) power-of-two scalings of the rows of ``A_s`` and the columns of
  ``B_s`` (Fig. 2), and ``E_s^-1 T F_s^-1`` is added to ``C``.

Readings (each also used by the GPU planner):

* "height of a row below 2^h" is ``max_k top(a_ik) - min_k bottom(a_ik) <= h`` over the nonzero
  entries, where ``top`` is the exponent ``e`` with ``2^(e-1) <= |a| < 2^e`` and ``bottom`` the
  exponent of the lowest set bit; the same for the columns of ``B``.
* The greedy search stops before the first index that breaks the bound.  When the first index
  alone breaks it (an entry taller than h, which happens when p < p_A), the block is that one
  index, so a block always holds at least one index and no full block ever exceeds h.
* ``h`` is rounded down to an integer.
* ``F_s`` scales column ``j`` (the figure's ``f_{i,s}`` index is read as ``f_{j,s}``).
* All contributions to an entry are summed exactly and rounded once, so a product without basecase
  blocks has the midpoint ``RNE_p(sum_k a_ik b_kj)``.

``plan_ordered`` / ``scaled_block_ordered`` restate Section IV-B's suggested improvement (an inner
scaling of the columns of A_s against the rows of B_s, combined with a permutation of the inner
index); its reading is given above ``inner_order``.  ``plan_complex_shared`` /
``scaled_block_complex`` / ``eq2_block_products`` restate Section IV-C's complex product by eq. 2
over blocks planned for both parts together; ``plan_complex_ordered`` /
``scaled_block_complex_ordered`` combine that with the inner ordering.  ``omission_thresholds``
/ ``omitted_product`` restate the negligible-limb omission of Section IV-B's last paragraph for a
real product, ``omission_thresholds_complex`` / ``omitted_product_complex`` for the two parts of a
complex product by eq. 2 under thresholds shared by the parts.
"""
from __future__ import annotations

from .exact import FLAG_SIGN, FLAG_ZERO, limb_field

BASECASE = 30


def top_bottom(raw, i):
    """``(top, bottom, signed_integer_mantissa, shift)`` of entry ``i``, or None if zero.

    The value is ``mant * 2^shift`` with ``mant`` odd; ``bottom = shift`` and ``top`` is the exponent
    of the entry."""
    fl = int(raw.flags[i])
    if fl & FLAG_ZERO:
        return None
    v = limb_field(raw, i)
    tz = (v & -v).bit_length() - 1
    mant = v >> tz
    shift = int(raw.exp[i]) - 64 * raw.nlimbs + tz
    if fl & FLAG_SIGN:
        mant = -mant
    return int(raw.exp[i]), shift, mant, shift


def precision_of(raw, count):
    """``p_M``: the largest ``top - bottom`` over the nonzero entries (0 for a zero matrix)."""
    best = 0
    for i in range(count):
        tb = top_bottom(raw, i)
        if tb is not None:
            best = max(best, tb[0] - tb[1])
    return best


def height_bound(prec, pA, pB):
    return (5 * min(prec, max(pA, pB))) // 4 + 192


def plan(A, B, M, K, N, prec):
    """Greedy block list ``[(start, stop, is_basecase)]`` over the inner dimension."""
    pA = precision_of(A, M * K)
    pB = precision_of(B, K * N)
    h = height_bound(prec, pA, pB)
    tbA = [[top_bottom(A, i * K + k) for k in range(K)] for i in range(M)]
    tbB = [[top_bottom(B, k * N + j) for k in range(K)] for j in range(N)]
    return h, _greedy(tbA, tbB, M, N, K, h)


def _greedy(tbA, tbB, M, N, K, h):
    """The greedy extraction over positions 0..K-1 of the per-line entry lists ``tbA[i][t]``,
    ``tbB[j][t]`` (``(top, bottom, ...)`` or None for a zero)."""
    blocks = []
    start = 0
    while start < K:
        stop = start + 1
        hi_a = [None] * M
        lo_a = [None] * M
        hi_b = [None] * N
        lo_b = [None] * N

        def admit(k):
            nha, nla, nhb, nlb = list(hi_a), list(lo_a), list(hi_b), list(lo_b)
            for i in range(M):
                tb = tbA[i][k]
                if tb is not None:
                    nha[i] = tb[0] if nha[i] is None else max(nha[i], tb[0])
                    nla[i] = tb[1] if nla[i] is None else min(nla[i], tb[1])
                    if nha[i] - nla[i] > h:
                        return None
            for j in range(N):
                tb = tbB[j][k]
                if tb is not None:
                    nhb[j] = tb[0] if nhb[j] is None else max(nhb[j], tb[0])
                    nlb[j] = tb[1] if nlb[j] is None else min(nlb[j], tb[1])
                    if nhb[j] - nlb[j] > h:
                        return None
            return nha, nla, nhb, nlb

        st = admit(start)
        if st is not None:
            hi_a, lo_a, hi_b, lo_b = st
            while stop < K:
                st = admit(stop)
                if st is None:
                    break
                hi_a, lo_a, hi_b, lo_b = st
                stop += 1
        # else: the first index alone breaks the bound (an entry taller than h, e.g. p_A > h);
        # the block is that index alone, so every block holds at least one index
        if stop - start < BASECASE:
            stop = start + min(BASECASE, K - start)
            blocks.append((start, stop, True))
        else:
            blocks.append((start, stop, False))
        start = stop
    return blocks


def scaled_block(A, B, M, K, N, start, stop):
    """``(e, f, X, Y)``: row exponents ``e_i``, column exponents ``f_j`` and the integer matrices
    ``X = E_s A_s`` (M x |s|) and ``Y = B_s F_s`` (|s| x N) of block ``[start, stop)`` (Fig. 2)."""
    e = []
    X = []
    for i in range(M):
        row = [top_bottom(A, i * K + k) for k in range(start, stop)]
        lows = [tb[1] for tb in row if tb is not None]
        ei = -min(lows) if lows else 0
        e.append(ei)
        X.append([0 if tb is None else tb[2] << (tb[3] + ei) for tb in row])
    f = []
    cols = []
    for j in range(N):
        col = [top_bottom(B, k * N + j) for k in range(start, stop)]
        lows = [tb[1] for tb in col if tb is not None]
        fj = -min(lows) if lows else 0
        f.append(fj)
        cols.append([0 if tb is None else tb[2] << (tb[3] + fj) for tb in col])
    Y = [[cols[j][kk] for j in range(N)] for kk in range(stop - start)]
    return e, f, X, Y


# ---- Section IV-B's suggested improvement: an inner scaling G_s G_s^-1 of the columns of A_s and
# the rows of B_s, combined with a permutation of the inner index (non-contiguous blocks).
#
# Reading (the paper leaves the strategy open; the GPU planner follows the same rule):
# * a_k = largest top over column k of A, b_k = largest top over row k of B;
# * an index whose column of A or row of B is entirely zero contributes nothing to the midpoint
#   product A B; it keeps g_k = 0 and comes after the live indices, in index order (its radii may
#   still count, so it is not dropped);
# * g_k = floor((b_k - a_k) / 2): column k of A is multiplied by 2^g_k and row k of B by 2^-g_k
#   (exact, and A B is unchanged), which brings both tops to within one of (a_k + b_k) / 2;
# * the live indices are ordered by a_k + b_k, the magnitude bound of their products (ties by
#   index), and the greedy extraction of Section IV-A runs over that order.

def inner_order(A, B, M, K, N):
    """``(order, g)``: a permutation of the inner indices in planning order (the live ones by
    a_k + b_k, then the dead ones) and the inner scaling exponent of every index (0 when dead)."""
    g = [0] * K
    keyed, dead = [], []
    for k in range(K):
        ta = [top_bottom(A, i * K + k) for i in range(M)]
        tb = [top_bottom(B, k * N + j) for j in range(N)]
        ta = [t[0] for t in ta if t is not None]
        tb = [t[0] for t in tb if t is not None]
        if not ta or not tb:
            dead.append(k)
            continue
        a, b = max(ta), max(tb)
        g[k] = (b - a) // 2
        keyed.append((a + b, k))
    keyed.sort()
    return [k for _, k in keyed] + dead, g


def plan_ordered(A, B, M, K, N, prec):
    """``(h, order, g, blocks)``: the greedy blocks over positions of ``order`` (blocks index
    positions; position t is inner index order[t]), under the inner scaling ``g``."""
    pA = precision_of(A, M * K)
    pB = precision_of(B, K * N)
    h = height_bound(prec, pA, pB)
    order, g = inner_order(A, B, M, K, N)

    def shifted(tb, d):
        return None if tb is None else (tb[0] + d, tb[1] + d, tb[2], tb[3] + d)
    tbA = [[shifted(top_bottom(A, i * K + k), g[k]) for k in order] for i in range(M)]
    tbB = [[shifted(top_bottom(B, k * N + j), -g[k]) for k in order] for j in range(N)]
    return h, order, g, _greedy(tbA, tbB, M, N, len(order), h)


def scaled_block_ordered(A, B, M, K, N, ks, g):
    """``(e, f, X, Y)`` of the block of inner indices ``ks`` (any order) under the inner scaling
    ``g``: ``X = E_s A_s G_s`` (M x |s|) and ``Y = G_s^-1 B_s F_s`` (|s| x N) with minimal-height
    row and column scalings (Fig. 2), so that ``E_s^-1 X Y F_s^-1 = A_s B_s``."""
    e, X = [], []
    for i in range(M):
        row = [top_bottom(A, i * K + k) for k in ks]
        sh = [None if tb is None else tb[3] + g[k] for tb, k in zip(row, ks)]
        lows = [v for v in sh if v is not None]
        ei = -min(lows) if lows else 0
        e.append(ei)
        X.append([0 if tb is None else tb[2] << (v + ei) for tb, v in zip(row, sh)])
    f, cols = [], []
    for j in range(N):
        col = [top_bottom(B, k * N + j) for k in ks]
        sh = [None if tb is None else tb[3] - g[k] for tb, k in zip(col, ks)]
        lows = [v for v in sh if v is not None]
        fj = -min(lows) if lows else 0
        f.append(fj)
        cols.append([0 if tb is None else tb[2] << (v + fj) for tb, v in zip(col, sh)])
    Y = [[cols[j][t] for j in range(N)] for t in range(len(ks))]
    return e, f, X, Y


# ---- Complex products by eq. 2 with several blocks (Section IV-C's second suggestion: a splitting
# and scaling strategy that considers the real and imaginary parts together).
#
# Reading: the height of a row of A_s (a column of B_s) is taken over both parts, so each entry
# contributes the larger top and the smaller bottom of its real and imaginary part; the greedy
# extraction of Section IV-A runs on those merged values, and each full block takes one scaling
# per row and per column for both parts.  Then X_re + X_im and Y_re + Y_im are integers and, per
# block, Re = P1 - P2 and Im = P3 - P1 - P2 with P1 = X_re Y_re, P2 = X_im Y_im,
# P3 = (X_re + X_im)(Y_re + Y_im) (eq. 2), all exact.

def _merged_tb(re, im, idx):
    a, b = top_bottom(re, idx), top_bottom(im, idx)
    if a is None and b is None:
        return None
    if a is None or b is None:
        t = a if a is not None else b
        return t[0], t[1]
    return max(a[0], b[0]), min(a[1], b[1])


def plan_complex_shared(A, B, M, K, N, prec):
    """``(h, blocks)`` for the complex product of ``A = (A_re, A_im)`` and ``B = (B_re, B_im)``
    with the merged heights; h from the largest precision over all four parts."""
    pA = max(precision_of(A[0], M * K), precision_of(A[1], M * K))
    pB = max(precision_of(B[0], K * N), precision_of(B[1], K * N))
    h = height_bound(prec, pA, pB)
    tbA = [[_merged_tb(A[0], A[1], i * K + k) for k in range(K)] for i in range(M)]
    tbB = [[_merged_tb(B[0], B[1], k * N + j) for k in range(K)] for j in range(N)]
    return h, _greedy(tbA, tbB, M, N, K, h)


def scaled_block_complex(A, B, M, K, N, start, stop):
    """``(e, f, (X_re, X_im), (Y_re, Y_im))`` of block ``[start, stop)`` under one minimal scaling
    per row of A and per column of B shared by both parts."""
    e = []
    Xs = ([], [])
    for i in range(M):
        rows = [[top_bottom(A[q], i * K + k) for k in range(start, stop)] for q in (0, 1)]
        lows = [tb[3] for row in rows for tb in row if tb is not None]
        ei = -min(lows) if lows else 0
        e.append(ei)
        for q in (0, 1):
            Xs[q].append([0 if tb is None else tb[2] << (tb[3] + ei) for tb in rows[q]])
    f = []
    cols = ([], [])
    for j in range(N):
        cs = [[top_bottom(B[q], k * N + j) for k in range(start, stop)] for q in (0, 1)]
        lows = [tb[3] for col in cs for tb in col if tb is not None]
        fj = -min(lows) if lows else 0
        f.append(fj)
        for q in (0, 1):
            cols[q].append([0 if tb is None else tb[2] << (tb[3] + fj) for tb in cs[q]])
    Ys = tuple([[cols[q][j][t] for j in range(N)] for t in range(stop - start)] for q in (0, 1))
    return e, f, Xs, Ys


# The two suggestions together: eq. 2 over blocks planned for both parts at once, over an inner
# order and scaling shared by the parts.  Reading: a_k is the largest top over column k of both
# parts of A, b_k over row k of both parts of B; g_k, the dead indices and the order follow
# ``inner_order``; the greedy extraction runs on the merged tops and bottoms of ``plan_complex_shared``
# shifted by g_k (column k of both parts of A) and -g_k (row k of both parts of B).

def inner_order_complex(A, B, M, K, N):
    """``(order, g)`` of ``inner_order`` with the tops merged over the real and imaginary parts."""
    g = [0] * K
    keyed, dead = [], []
    for k in range(K):
        ta = [t[0] for q in (0, 1) for t in (top_bottom(A[q], i * K + k) for i in range(M))
              if t is not None]
        tb = [t[0] for q in (0, 1) for t in (top_bottom(B[q], k * N + j) for j in range(N))
              if t is not None]
        if not ta or not tb:
            dead.append(k)
            continue
        a, b = max(ta), max(tb)
        g[k] = (b - a) // 2
        keyed.append((a + b, k))
    keyed.sort()
    return [k for _, k in keyed] + dead, g


def plan_complex_ordered(A, B, M, K, N, prec):
    """``(h, order, g, blocks)``: the merged-part greedy blocks over positions of the shared order
    under the shared inner scaling (h as in ``plan_complex_shared``)."""
    pA = max(precision_of(A[0], M * K), precision_of(A[1], M * K))
    pB = max(precision_of(B[0], K * N), precision_of(B[1], K * N))
    h = height_bound(prec, pA, pB)
    order, g = inner_order_complex(A, B, M, K, N)

    def shifted(tb, d):
        return None if tb is None else (tb[0] + d, tb[1] + d)
    tbA = [[shifted(_merged_tb(A[0], A[1], i * K + k), g[k]) for k in order] for i in range(M)]
    tbB = [[shifted(_merged_tb(B[0], B[1], k * N + j), -g[k]) for k in order] for j in range(N)]
    return h, order, g, _greedy(tbA, tbB, M, N, len(order), h)


def scaled_block_complex_ordered(A, B, M, K, N, ks, g):
    """``(e, f, (X_re, X_im), (Y_re, Y_im))`` of the block of inner indices ``ks`` under the inner
    scaling ``g``: ``X_q = E_s A_q,s G_s`` and ``Y_q = G_s^-1 B_q,s F_s`` with one minimal scaling
    per row of A and per column of B shared by both parts."""
    e = []
    Xs = ([], [])
    for i in range(M):
        rows = [[top_bottom(A[q], i * K + k) for k in ks] for q in (0, 1)]
        sh = [[None if tb is None else tb[3] + g[k] for tb, k in zip(rows[q], ks)] for q in (0, 1)]
        lows = [v for q in (0, 1) for v in sh[q] if v is not None]
        ei = -min(lows) if lows else 0
        e.append(ei)
        for q in (0, 1):
            Xs[q].append([0 if tb is None else tb[2] << (v + ei) for tb, v in zip(rows[q], sh[q])])
    f = []
    cols = ([], [])
    for j in range(N):
        cs = [[top_bottom(B[q], k * N + j) for k in ks] for q in (0, 1)]
        sh = [[None if tb is None else tb[3] - g[k] for tb, k in zip(cs[q], ks)] for q in (0, 1)]
        lows = [v for q in (0, 1) for v in sh[q] if v is not None]
        fj = -min(lows) if lows else 0
        f.append(fj)
        for q in (0, 1):
            cols[q].append([0 if tb is None else tb[2] << (v + fj) for tb, v in zip(cs[q], sh[q])])
    Ys = tuple([[cols[q][j][t] for j in range(N)] for t in range(len(ks))] for q in (0, 1))
    return e, f, Xs, Ys


def eq2_block_products(Xs, Ys):
    """``(Re, Im)`` of one block from three integer products (eq. 2)."""
    Xr, Xi = Xs
    Yr, Yi = Ys
    P1 = int_matmul(Xr, Yr)
    P2 = int_matmul(Xi, Yi)
    Xsum = [[a + b for a, b in zip(ra, rb)] for ra, rb in zip(Xr, Xi)]
    Ysum = [[a + b for a, b in zip(ra, rb)] for ra, rb in zip(Yr, Yi)]
    P3 = int_matmul(Xsum, Ysum)
    Re = [[p1 - p2 for p1, p2 in zip(r1, r2)] for r1, r2 in zip(P1, P2)]
    Im = [[p3 - p1 - p2 for p3, p1, p2 in zip(r3, r1, r2)] for r3, r1, r2 in zip(P3, P1, P2)]
    return Re, Im


def int_matmul(X, Y):
    """Textbook integer matrix product on Python integers."""
    n_in = len(Y)
    N = len(Y[0]) if n_in else 0
    return [[sum(row[k] * Y[k][j] for k in range(n_in)) for j in range(N)] for row in X]


def int_matmul_entry(X, Y, i, j):
    return sum(X[i][k] * Y[k][j] for k in range(len(Y)))


def height(v: int) -> int:
    return abs(v).bit_length()


# ---- Section IV-B's last paragraph: Algorithm 2 uses every input bit, where Algorithm 1 omits
# negligible limbs.  Reading (the paper leaves it to future work; the GPU path follows the same
# rule): with E_ij = max_k top(a_ik) + top(b_kj) (the largest product exponent of entry (i, j),
# Algorithm 1's e_max of that dot), every bit of row i of A below 2^tau_i and of column j of B
# below 2^sigma_j is dropped (truncation toward zero), where
#     tau_i = min_j (E_ij - top_j(B)) - p - G,   sigma_j = min_i (E_ij - top_i(A)) - p - G,
#     G = bc(K) + 8,
# the minima over the entries with a nonzero product.  Then |a_ik - a'_ik| < 2^tau_i and the
# error of every product sum is below K (2^(tau_i + top_j) + 2^(top_i + sigma_j) + ...) <=
# 3 K 2^(E_ij - p - G) < 2^-p 2^(E_ij - 2) 3/64 <= (3/64) 2^-p sum_k |a_ik b_kj|; each truncated
# line's nonzero entries carry 2^tau (2^sigma) more radius, so the ball stays rigorous.  A line
# without any nonzero product is left as it is.

def bc(v: int) -> int:
    return int(v).bit_length()


def omission_thresholds(A, B, M, K, N, prec):
    """``(tau, sigma)``: the truncation exponents of the rows of A and the columns of B (None for a
    line left as it is)."""
    G = bc(K) + 8
    ta = [[top_bottom(A, i * K + k) for k in range(K)] for i in range(M)]
    tb = [[top_bottom(B, k * N + j) for j in range(N)] for k in range(K)]
    rtop = [max((t[0] for t in row if t is not None), default=None) for row in ta]
    ctop = [max((tb[k][j][0] for k in range(K) if tb[k][j] is not None), default=None)
            for j in range(N)]
    E = [[None] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            for k in range(K):
                a, b = ta[i][k], tb[k][j]
                if a is not None and b is not None:
                    v = a[0] + b[0]
                    E[i][j] = v if E[i][j] is None else max(E[i][j], v)
    tau = []
    for i in range(M):
        d = [E[i][j] - ctop[j] for j in range(N) if E[i][j] is not None]
        tau.append(min(d) - prec - G if d else None)
    sigma = []
    for j in range(N):
        d = [E[i][j] - rtop[i] for i in range(M) if E[i][j] is not None]
        sigma.append(min(d) - prec - G if d else None)
    return tau, sigma


def truncate_value(tb, t):
    """The value ``mant 2^shift`` of ``tb = top_bottom(...)`` with every bit below 2^t dropped
    (toward zero), as ``(integer, exponent)``; ``t`` None keeps it."""
    if tb is None:
        return 0, 0
    mant, shift = tb[2], tb[3]
    if t is None or shift >= t:
        return mant, shift
    q = abs(mant) >> (t - shift)
    return (q if mant > 0 else -q), t


def omitted_product(A, B, M, K, N, tau, sigma):
    """The exact product of the truncated operands, entry by entry, as Fractions."""
    from fractions import Fraction
    a = [[truncate_value(top_bottom(A, i * K + k), tau[i]) for k in range(K)] for i in range(M)]
    b = [[truncate_value(top_bottom(B, k * N + j), sigma[j]) for j in range(N)]
         for k in range(K)]

    def val(v):
        return Fraction(v[0]) * Fraction(2) ** v[1]
    return [[sum(val(a[i][k]) * val(b[k][j]) for k in range(K)) for j in range(N)]
            for i in range(M)]


# ---- the omission for eq. 2 (Section IV-B's last paragraph with Section IV-C's shared scaling).
# Reading: both parts of a row of A (a column of B) drop their bits below one threshold, so the
# truncated parts still take one scaling per line shared by both parts.  With E_q,ij the largest
# product exponent of output part q at (i, j) (q = 0: a_re b_re and a_im b_im; q = 1: a_re b_im
# and a_im b_re), rtop_i / ctop_j the line tops over both parts, and G = bc(K) + 9,
#     tau_i = min_{q, j} (E_q,ij - ctop_j) - p - G,   sigma_j = min_{q, i} (E_q,ij - rtop_i) - p - G
# (minima over the (q, i, j) with a nonzero product).  Each of part q's 2 K products then changes
# by less than 2^(tau_i + ctop_j) + 2^(rtop_i + sigma_j) <= 2 2^(E_q,ij - p - G), so part q changes
# by less than 4 K 2^(E_q,ij - p - G) < 2^(E_q,ij - 2) 2^-p / 32 <= (1/32) 2^-p times the sum of
# |a b| over part q's terms: one bit more of G than a real product takes, for the two products
# each part sums.  The bound of each part is its own: a threshold taken from the larger part's E
# alone would drop bits that matter to the smaller part.

def omission_thresholds_complex(A, B, M, K, N, prec):
    """``(tau, sigma)`` shared by both parts of ``A = (A_re, A_im)`` and ``B = (B_re, B_im)`` (None
    for a line left as it is)."""
    G = bc(K) + 9
    ta = [[[top_bottom(A[q], i * K + k) for k in range(K)] for i in range(M)] for q in (0, 1)]
    tb = [[[top_bottom(B[q], k * N + j) for j in range(N)] for k in range(K)] for q in (0, 1)]
    rtop = [max((t[0] for q in (0, 1) for t in ta[q][i] if t is not None), default=None)
            for i in range(M)]
    ctop = [max((tb[q][k][j][0] for q in (0, 1) for k in range(K) if tb[q][k][j] is not None),
                default=None) for j in range(N)]
    products = (((0, 0), (1, 1)), ((0, 1), (1, 0)))  # (A part, B part) of Re, then of Im
    E = [[[None] * N for _ in range(M)] for _ in products]
    for part, pairs in enumerate(products):
        for i in range(M):
            for j in range(N):
                for x, y in pairs:
                    for k in range(K):
                        a, b = ta[x][i][k], tb[y][k][j]
                        if a is not None and b is not None:
                            v = a[0] + b[0]
                            e = E[part][i][j]
                            E[part][i][j] = v if e is None else max(e, v)
    tau = []
    for i in range(M):
        d = [E[q][i][j] - ctop[j] for q in (0, 1) for j in range(N) if E[q][i][j] is not None]
        tau.append(min(d) - prec - G if d else None)
    sigma = []
    for j in range(N):
        d = [E[q][i][j] - rtop[i] for q in (0, 1) for i in range(M) if E[q][i][j] is not None]
        sigma.append(min(d) - prec - G if d else None)
    return tau, sigma


def omitted_product_complex(A, B, M, K, N, tau, sigma):
    """``(Re, Im)`` of the exact complex product of the truncated parts, entry by entry, as
    Fractions."""
    P = {(x, y): omitted_product(A[x], B[y], M, K, N, tau, sigma) for x in (0, 1) for y in (0, 1)}
    re = [[P[0, 0][i][j] - P[1, 1][i][j] for j in range(N)] for i in range(M)]
    im = [[P[0, 1][i][j] + P[1, 0][i][j] for j in range(N)] for i in range(M)]
    return re, im
