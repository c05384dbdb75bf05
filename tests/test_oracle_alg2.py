"""Pins for the Algorithm 2 restatement (``oracle.alg2``): the block decomposition must reproduce the
exact product (checked with ``fractions.Fraction`` arithmetic), the integer product must agree with
numpy's integer matmul, the scalings must be minimal, the greedy blocks maximal, and the height bound
must follow the paper's formula."""
from __future__ import annotations

import math
import zlib
from fractions import Fraction

import numpy as np
import pytest

from oracle import alg2
from oracle import exact as X
from synth import random_balls
from synth.workloads import matmul_uniform
from tests.ballmake import ball_values, make_balls


def exact_product(A, B, M, K, N):
    out = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            out[i][j] = sum(ball_values(A, i * K + k)[0] * ball_values(B, k * N + j)[0]
                            for k in range(K))
    return out


def recombined(A, B, M, K, N, prec):
    h, blocks = alg2.plan(A, B, M, K, N, prec)
    C = [[Fraction(0)] * N for _ in range(M)]
    for start, stop, base in blocks:
        if base:
            for i in range(M):
                for j in range(N):
                    C[i][j] += sum(ball_values(A, i * K + k)[0] * ball_values(B, k * N + j)[0]
                                   for k in range(start, stop))
        else:
            e, f, Xs, Ys = alg2.scaled_block(A, B, M, K, N, start, stop)
            T = alg2.int_matmul(Xs, Ys)
            for i in range(M):
                for j in range(N):
                    C[i][j] += Fraction(T[i][j]) * Fraction(2) ** (-e[i] - f[j])
    return h, blocks, C


@pytest.mark.parametrize("kind", ["uniform", "badly_scaled", "zeros", "short"])
def test_blocks_reproduce_exact_product(kind):
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    if kind == "uniform":
        M, K, N, p = 3, 40, 4, 128
        A = random_balls(rng, M * K, 2, 128, -20, 20)
        B = random_balls(rng, K * N, 2, 128, -20, 20)
    elif kind == "badly_scaled":
        M, K, N, p = 3, 70, 2, 64
        ea = rng.integers(-5, 5, size=M * K)
        ea[np.arange(M) * K + 35] += 900  # column 35 of A is 2^900 larger: forces a split
        A = random_balls(rng, M * K, 1, 64, exps=ea)
        B = random_balls(rng, K * N, 1, 64, -5, 5)
    elif kind == "zeros":
        M, K, N, p = 2, 35, 3, 64
        A = random_balls(rng, M * K, 1, 64, -5, 5, zero_frac=0.4)
        B = random_balls(rng, K * N, 1, 64, -5, 5, zero_frac=0.4)
        A.flags[0:K] = X.FLAG_ZERO  # row 0 of A entirely zero
        A.limbs[:, 0:K] = 0
    else:
        M, K, N, p = 2, 12, 2, 64
        A = random_balls(rng, M * K, 1, 64, -5, 5)
        B = random_balls(rng, K * N, 1, 64, -5, 5)
    h, blocks, C = recombined(A, B, M, K, N, p)
    assert C == exact_product(A, B, M, K, N)
    # the blocks tile [0, K) in order
    assert blocks[0][0] == 0 and blocks[-1][1] == K
    assert all(blocks[t][1] == blocks[t + 1][0] for t in range(len(blocks) - 1))
    if kind == "uniform":
        assert blocks == [(0, K, False)]
    if kind == "short":
        assert blocks == [(0, K, True)]
    if kind == "badly_scaled":
        assert len(blocks) >= 2


def test_height_bound_formula():
    for p, pa, pb in [(256, 256, 256), (128, 128, 128), (53, 53, 53), (1024, 300, 2000),
                      (106, 53, 64)]:
        assert alg2.height_bound(p, pa, pb) == math.floor(1.25 * min(p, max(pa, pb)) + 192)
    assert alg2.height_bound(256, 256, 256) == 512
    assert alg2.height_bound(128, 128, 128) == 352


def test_precision_of_matrix():
    A = make_balls([Fraction(3, 4), Fraction(1, 2**10), Fraction(5)])
    # 3/4 = 11b * 2^-2 -> 2 bits; 2^-10 -> 1 bit; 5 = 101b -> 3 bits
    assert alg2.precision_of(A, 3) == 3


def test_scaling_is_minimal_and_integral():
    rng = np.random.default_rng(2)
    M, K, N = 4, 33, 3
    A = random_balls(rng, M * K, 2, 100, -30, 30)
    B = random_balls(rng, K * N, 2, 100, -30, 30)
    e, f, Xs, Ys = alg2.scaled_block(A, B, M, K, N, 0, K)
    for i in range(M):
        assert any(v & 1 for v in Xs[i])  # minimal: some entry odd
        for k in range(K):
            assert Fraction(Xs[i][k]) == ball_values(A, i * K + k)[0] * Fraction(2) ** e[i]
    for j in range(N):
        assert any(Ys[k][j] & 1 for k in range(K))
        for k in range(K):
            assert Fraction(Ys[k][j]) == ball_values(B, k * N + j)[0] * Fraction(2) ** f[j]


def _greedy_case(drift):
    """Two rows of A against a narrow B.  Without drift the exponents of A are i.i.d. over a range
    wider than h, so every block is a basecase block; with drift they climb 6 per inner index, so
    full blocks of about 34 indices form and each ends before K."""
    rng = np.random.default_rng(3)
    M, K, N, p = 2, 150, 2, 64
    if drift:
        ea = np.repeat(6 * np.arange(K)[None, :], M, axis=0).ravel() + rng.integers(-3, 4, M * K)
    else:
        ea = rng.integers(-200, 200, size=M * K)
    A = random_balls(rng, M * K, 1, 64, exps=ea)
    B = random_balls(rng, K * N, 1, 64, -3, 3)
    return A, B, M, K, N, p


def _check_greedy(A, B, M, K, N, h, blocks):
    def height_ok(start, stop):
        for i in range(M):
            tbs = [alg2.top_bottom(A, i * K + k) for k in range(start, stop)]
            if max(t[0] for t in tbs) - min(t[1] for t in tbs) > h:
                return False
        for j in range(N):
            tbs = [alg2.top_bottom(B, k * N + j) for k in range(start, stop)]
            if max(t[0] for t in tbs) - min(t[1] for t in tbs) > h:
                return False
        return True

    assert blocks[0][0] == 0 and blocks[-1][1] == K
    assert all(blocks[t][1] == blocks[t + 1][0] for t in range(len(blocks) - 1))
    for start, stop, base in blocks:
        if not base:
            assert stop - start >= alg2.BASECASE
            assert height_ok(start, stop)
            if stop < K:
                assert not height_ok(start, stop + 1)  # maximal
        else:  # a basecase block: the greedy block from `start` is shorter than 30 indices
            t = start + 1
            while t < K and height_ok(start, t + 1):
                t += 1
            assert t - start < alg2.BASECASE


@pytest.mark.parametrize("drift", [False, True])
def test_greedy_blocks_are_within_height_and_maximal(drift):
    A, B, M, K, N, p = _greedy_case(drift)
    h, blocks = alg2.plan(A, B, M, K, N, p)
    _check_greedy(A, B, M, K, N, h, blocks)
    if drift:  # the maximality check above really ran
        assert any(not base and stop < K for _, stop, base in blocks)
    else:
        assert all(base for _, _, base in blocks)


def _brute_plan(A, B, M, K, N, h):
    """The plan rule written out by brute force: from each start, the longest range [start, t) in
    which every row of A and column of B (heights recomputed from scratch for every range) has
    height <= h, but at least one index; a range shorter than 30 is widened to min(30, K - start)
    and marked as a basecase block."""
    def line_ok(tbs):
        tbs = [t for t in tbs if t is not None]
        return not tbs or max(t[0] for t in tbs) - min(t[1] for t in tbs) <= h

    def ok(start, stop):
        return (all(line_ok([alg2.top_bottom(A, i * K + k) for k in range(start, stop)])
                    for i in range(M)) and
                all(line_ok([alg2.top_bottom(B, k * N + j) for k in range(start, stop)])
                    for j in range(N)))
    out, start = [], 0
    while start < K:
        t = start
        while t < K and ok(start, t + 1):
            t += 1
        stop = max(t, start + 1)
        if stop - start < alg2.BASECASE:
            stop = start + min(alg2.BASECASE, K - start)
            out.append((start, stop, True))
        else:
            out.append((start, stop, False))
        start = stop
    return out


def _tall_case(kind):
    """Products at p = 64 with some 1024-bit entries: p_A > p makes h = 1.25*64 + 192 = 272, so a
    1024-bit entry alone is taller than h and its index can only form a block by itself."""
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    if kind == "all_tall":       # every entry is taller than h
        M, K, N = 2, 40, 2
        bits_a = np.full(M * K, 1024)
    elif kind == "tall_then_zeros":  # row 0 of A: a tall entry at index 0, zeros after it
        M, K, N = 3, 70, 2
        bits_a = np.full(M * K, 64)
        bits_a[0] = 1024
    else:                        # "tall_in_middle": one tall entry at index 40 of row 1
        M, K, N = 2, 100, 3
        bits_a = np.full(M * K, 64)
        bits_a[K + 40] = 1024
    A = random_balls(rng, M * K, 16, bits_a, -5, 5)
    B = random_balls(rng, K * N, 16, 64, -5, 5)
    if kind == "tall_then_zeros":
        A.limbs[:, 1:K] = 0
        A.flags[1:K] = X.FLAG_ZERO
        A.exp[1:K] = 0
    return A, B, M, K, N, 64


TALL_PLANS = {
    "all_tall": [(0, 30, True), (30, 40, True)],
    "tall_then_zeros": [(0, 30, True), (30, 70, False)],
    "tall_in_middle": [(0, 40, False), (40, 70, True), (70, 100, False)],
}


@pytest.mark.parametrize("kind", sorted(TALL_PLANS))
def test_entry_taller_than_h_forms_a_block_alone(kind):
    """Section IV-A's greedy extraction when an entry is taller than h (p < p_A): the index of such
    an entry is a block by itself (then widened to a basecase block), every block holds at least
    one index, the plan equals the brute-force rule, and the blocks reproduce the exact product."""
    A, B, M, K, N, p = _tall_case(kind)
    h, blocks, C = recombined(A, B, M, K, N, p)
    assert h == 272
    assert blocks == TALL_PLANS[kind] == _brute_plan(A, B, M, K, N, h)
    assert all(stop > start for start, stop, _ in blocks)
    assert C == exact_product(A, B, M, K, N)


def test_extending_a_forced_block_is_caught():
    """A planted variant of the rule that keeps growing a block whose first index is taller than h
    (while the next indices leave the tall lines empty) gives a different plan, which the
    brute-force pin above rejects."""
    A, B, M, K, N, p = _tall_case("tall_then_zeros")
    h = 272

    def tall_line_touched(start, k):
        for i in range(M):
            tbs = [alg2.top_bottom(A, i * K + t) for t in range(start, k + 1)]
            if tbs[-1] is not None:
                live = [t for t in tbs if t is not None]
                if max(t[0] for t in live) - min(t[1] for t in live) > h:
                    return True
        for j in range(N):
            tbs = [alg2.top_bottom(B, t * N + j) for t in range(start, k + 1)]
            if tbs[-1] is not None:
                live = [t for t in tbs if t is not None]
                if max(t[0] for t in live) - min(t[1] for t in live) > h:
                    return True
        return False
    stop = 1
    while stop < K and not tall_line_touched(0, stop):
        stop += 1
    planted = [(0, stop, stop < alg2.BASECASE)]
    assert planted == [(0, K, False)]
    assert planted != _brute_plan(A, B, M, K, N, h)
    assert alg2.plan(A, B, M, K, N, p)[1] == _brute_plan(A, B, M, K, N, h)


def test_int_matmul_vs_numpy():
    rng = np.random.default_rng(4)
    Xm = rng.integers(-2**20, 2**20, size=(5, 7))
    Ym = rng.integers(-2**20, 2**20, size=(7, 3))
    T = alg2.int_matmul(Xm.tolist(), Ym.tolist())
    assert T == (Xm.astype(np.int64) @ Ym.astype(np.int64)).tolist()


def test_uniform_workload_is_one_block():
    case = matmul_uniform(9, 40, 256, -20, 20, rad_bits=250)
    h, blocks = alg2.plan(case.A[0], case.B[0], 40, 40, 40, 256)
    assert h == 512 and blocks == [(0, 40, False)]


# ------------------------------------------------------------------ planted mistakes

def _fails(fn, *args):
    try:
        fn(*args)
    except (AssertionError, IndexError, ValueError):
        return True
    return False


def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the restatement makes at least one pin above fail."""
    orig_tb, orig_sb, orig_plan = alg2.top_bottom, alg2.scaled_block, alg2.plan

    # (a) the sign of a mantissa dropped: the blocks no longer reproduce the exact product
    def unsigned(raw, i):
        r = orig_tb(raw, i)
        return None if r is None else (r[0], r[1], abs(r[2]), r[3])
    monkeypatch.setattr(alg2, "top_bottom", unsigned)
    assert _fails(test_blocks_reproduce_exact_product, "uniform")
    monkeypatch.setattr(alg2, "top_bottom", orig_tb)

    # (b) the lowest set bit placed one position too high: every value doubles
    def shifted(raw, i):
        r = orig_tb(raw, i)
        return None if r is None else (r[0], r[1] + 1, r[2], r[3] + 1)
    monkeypatch.setattr(alg2, "top_bottom", shifted)
    assert _fails(test_blocks_reproduce_exact_product, "badly_scaled")
    monkeypatch.setattr(alg2, "top_bottom", orig_tb)

    # (c) a scaling one bit larger than needed: still exact, but no longer minimal (Fig. 2)
    def loose(A, B, M, K, N, start, stop):
        e, f, Xs, Ys = orig_sb(A, B, M, K, N, start, stop)
        return [v + 1 for v in e], f, [[2 * x for x in row] for row in Xs], Ys
    monkeypatch.setattr(alg2, "scaled_block", loose)
    assert not _fails(test_blocks_reproduce_exact_product, "uniform")
    assert _fails(test_scaling_is_minimal_and_integral)
    monkeypatch.setattr(alg2, "scaled_block", orig_sb)

    # (d) a transposed operand in the integer product
    monkeypatch.setattr(alg2, "int_matmul", lambda X, Y: [[sum(r[k] * Y[j][k] for k in range(len(r)))
                                                           for j in range(len(Y[0]))] for r in X])
    assert _fails(test_int_matmul_vs_numpy)
    monkeypatch.undo()

    # (e) the greedy search stopping one index early (the next block starting there)
    def early(A, B, M, K, N, prec):
        h, blocks = orig_plan(A, B, M, K, N, prec)
        out, shift = [], 0
        for start, stop, base in blocks:
            start -= shift
            if not base and stop < K:
                out.append((start, stop - 1, base))
                shift = 1
            else:
                out.append((start, stop, base))
                shift = 0
        return h, out
    A, B, M, K, N, p = _greedy_case(True)
    h, blocks = early(A, B, M, K, N, p)
    assert _fails(_check_greedy, A, B, M, K, N, h, blocks)
    h, blocks = orig_plan(A, B, M, K, N, p)
    assert not _fails(_check_greedy, A, B, M, K, N, h, blocks)


# ------------------------------------------------------------------ inner scaling + permutation
# (Section IV-B's suggested improvement, in the reading of ``oracle.alg2.inner_order``)

def recombined_ordered(A, B, M, K, N, prec):
    h, order, g, blocks = alg2.plan_ordered(A, B, M, K, N, prec)
    C = [[Fraction(0)] * N for _ in range(M)]
    for start, stop, base in blocks:
        ks = order[start:stop]
        if base:
            for i in range(M):
                for j in range(N):
                    C[i][j] += sum(ball_values(A, i * K + k)[0] * ball_values(B, k * N + j)[0]
                                   for k in ks)
        else:
            e, f, Xs, Ys = alg2.scaled_block_ordered(A, B, M, K, N, ks, g)
            T = alg2.int_matmul(Xs, Ys)
            for i in range(M):
                for j in range(N):
                    C[i][j] += Fraction(T[i][j]) * Fraction(2) ** (-e[i] - f[j])
    return order, g, blocks, C


def _ordered_case(kind):
    from synth.workloads import complex_matmul_laplace
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    if kind in ("structured", "literal"):
        case = complex_matmul_laplace(n=32, structured=(kind == "structured"))
        return case.A[0], case.B[1], 32, 32, 32, 128
    if kind == "uniform":
        M, K, N, p = 5, 36, 4, 128
        return (random_balls(rng, M * K, 2, 128, -20, 20), random_balls(rng, K * N, 2, 128, -20, 20),
                M, K, N, p)
    # zeros: column 3 of A and row 7 of B entirely zero, scattered zero entries elsewhere
    M, K, N, p = 4, 40, 3, 64
    A = random_balls(rng, M * K, 1, 64, -5, 5, zero_frac=0.3)
    B = random_balls(rng, K * N, 1, 64, -5, 5, zero_frac=0.3)
    for i in range(M):
        A.flags[i * K + 3] = X.FLAG_ZERO
        A.limbs[:, i * K + 3] = 0
    B.flags[7 * N:8 * N] = X.FLAG_ZERO
    B.limbs[:, 7 * N:8 * N] = 0
    return A, B, M, K, N, p


@pytest.mark.parametrize("kind", ["structured", "literal", "uniform", "zeros"])
def test_ordered_blocks_reproduce_exact_product(kind):
    A, B, M, K, N, p = _ordered_case(kind)
    order, g, blocks, C = recombined_ordered(A, B, M, K, N, p)
    assert C == exact_product(A, B, M, K, N)
    # the blocks tile the positions of the order, and the order is a set of distinct indices
    assert blocks[0][0] == 0 and blocks[-1][1] == len(order)
    assert all(blocks[t][1] == blocks[t + 1][0] for t in range(len(blocks) - 1))
    assert sorted(order) == list(range(K))  # a permutation of the inner indices
    if kind == "zeros":  # the dead indices (3, 7 and any that the random zeros emptied) last
        dead = [k for k in range(K) if not all(_tops(A, B, M, K, N, k))]
        assert {3, 7} <= set(dead) and order[K - len(dead):] == dead


def _tops(A, B, M, K, N, k):
    ta = [alg2.top_bottom(A, i * K + k) for i in range(M)]
    tb = [alg2.top_bottom(B, k * N + j) for j in range(N)]
    return [t[0] for t in ta if t], [t[0] for t in tb if t]


def test_inner_order_is_sorted_balanced_and_leaves_out_dead_indices():
    A, B, M, K, N, p = _ordered_case("zeros")
    order, g = alg2.inner_order(A, B, M, K, N)
    live = [k for k in range(K) if all(_tops(A, B, M, K, N, k))]
    dead = [k for k in range(K) if k not in live]
    assert sorted(order[:len(live)]) == live and order[len(live):] == dead
    assert all(g[k] == 0 for k in dead)
    keys = []
    for k in order[:len(live)]:
        ta, tb = _tops(A, B, M, K, N, k)
        a, b = max(ta), max(tb)
        keys.append(a + b)
        assert abs((a + g[k]) - (b - g[k])) <= 1  # the scaled tops meet in the middle
    assert keys == sorted(keys)


def test_ordered_greedy_blocks_are_within_height_and_maximal():
    from synth.workloads import complex_matmul_laplace
    case = complex_matmul_laplace(n=48, structured=True)
    A, B, M, K, N, p = case.A[0], case.B[0], 48, 48, 48, 128
    h, order, g, blocks = alg2.plan_ordered(A, B, M, K, N, p)

    def height_ok(start, stop):
        ks = order[start:stop]
        for i in range(M):
            tbs = [(t[0] + g[k], t[1] + g[k]) for k in ks
                   for t in [alg2.top_bottom(A, i * K + k)] if t]
            if tbs and max(t[0] for t in tbs) - min(t[1] for t in tbs) > h:
                return False
        for j in range(N):
            tbs = [(t[0] - g[k], t[1] - g[k]) for k in ks
                   for t in [alg2.top_bottom(B, k * N + j)] if t]
            if tbs and max(t[0] for t in tbs) - min(t[1] for t in tbs) > h:
                return False
        return True

    for start, stop, base in blocks:
        if not base:
            assert height_ok(start, stop)
            if stop < len(order):
                assert not height_ok(start, stop + 1)


def test_ordering_turns_the_structured_workload_into_full_blocks():
    """On the structured Laplace(40) workload at N = 128 the contiguous greedy leaves most of the
    inner dimension to basecase dots; ordered and scaled, nearly all of it forms full blocks."""
    from synth.workloads import complex_matmul_laplace
    n = 128
    case = complex_matmul_laplace(n=n, structured=True)
    for xa, yb in ((0, 0), (1, 1)):
        A, B = case.A[xa], case.B[yb]
        _, blocks = alg2.plan(A, B, n, n, n, 128)
        _, order, _, blocks2 = alg2.plan_ordered(A, B, n, n, n, 128)
        base1 = sum(b - a for a, b, base in blocks if base) / n
        base2 = sum(b - a for a, b, base in blocks2 if base) / n
        assert base1 >= 0.5 and base2 <= 0.1, (base1, base2)


def test_planted_mistakes_in_the_ordered_plan_are_caught(monkeypatch):
    orig = alg2.inner_order

    # (f) the inner scaling forgotten
    monkeypatch.setattr(alg2, "inner_order",
                        lambda A, B, M, K, N: (orig(A, B, M, K, N)[0], [0] * K))
    assert _fails(test_inner_order_is_sorted_balanced_and_leaves_out_dead_indices)
    monkeypatch.setattr(alg2, "inner_order", orig)

    # (g) ordered by the tops of A alone instead of the product bound a_k + b_k
    def by_a(A, B, M, K, N):
        order, g = orig(A, B, M, K, N)
        live = [k for k in order if all(_tops(A, B, M, K, N, k))]
        key = {k: max(_tops(A, B, M, K, N, k)[0]) for k in live}
        return sorted(live, key=lambda k: (key[k], k)) + order[len(live):], g
    monkeypatch.setattr(alg2, "inner_order", by_a)
    assert _fails(test_inner_order_is_sorted_balanced_and_leaves_out_dead_indices)
    monkeypatch.setattr(alg2, "inner_order", orig)
    assert not _fails(test_inner_order_is_sorted_balanced_and_leaves_out_dead_indices)


# ------------------------------------------------------------------ complex, eq. 2 over shared blocks
# (Section IV-C's second suggestion, in the reading of ``oracle.alg2.plan_complex_shared``)

def exact_complex_product(A, B, M, K, N):
    re = [[Fraction(0)] * N for _ in range(M)]
    im = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for j in range(N):
            for k in range(K):
                ar, ai = ball_values(A[0], i * K + k)[0], ball_values(A[1], i * K + k)[0]
                br, bi = ball_values(B[0], k * N + j)[0], ball_values(B[1], k * N + j)[0]
                re[i][j] += ar * br - ai * bi
                im[i][j] += ar * bi + ai * br
    return re, im


def recombined_complex(A, B, M, K, N, prec, products=alg2.eq2_block_products):
    h, blocks = alg2.plan_complex_shared(A, B, M, K, N, prec)
    re = [[Fraction(0)] * N for _ in range(M)]
    im = [[Fraction(0)] * N for _ in range(M)]
    for start, stop, base in blocks:
        if base:
            sub_re, sub_im = exact_complex_product(
                [_cols(A[q], M, K, start, stop) for q in (0, 1)],
                [_rows(B[q], K, N, start, stop) for q in (0, 1)], M, stop - start, N)
        else:
            e, f, Xs, Ys = alg2.scaled_block_complex(A, B, M, K, N, start, stop)
            R, I = products(Xs, Ys)
            sc = [[Fraction(2) ** (-e[i] - f[j]) for j in range(N)] for i in range(M)]
            sub_re = [[R[i][j] * sc[i][j] for j in range(N)] for i in range(M)]
            sub_im = [[I[i][j] * sc[i][j] for j in range(N)] for i in range(M)]
        for i in range(M):
            for j in range(N):
                re[i][j] += sub_re[i][j]
                im[i][j] += sub_im[i][j]
    return blocks, re, im


def _cols(raw, M, K, start, stop):
    idx = [i * K + k for i in range(M) for k in range(start, stop)]
    return _take(raw, idx)


def _rows(raw, K, N, start, stop):
    idx = [k * N + j for k in range(start, stop) for j in range(N)]
    return _take(raw, idx)


def _take(raw, idx):
    from synth import RawBalls
    idx = np.asarray(idx)
    return RawBalls(raw.nlimbs, raw.limbs[:, idx].copy(), raw.exp[idx].copy(),
                    raw.flags[idx].copy(), raw.rad_man[idx].copy(), raw.rad_exp[idx].copy())


def _complex_case(kind):
    from synth.workloads import complex_matmul_laplace
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    if kind == "structured":
        case = complex_matmul_laplace(n=32, structured=True)
        return case.A, case.B, 32, 32, 32, 128
    if kind == "banded":  # columns 40..79 of both parts of A sit 2^900 higher: two full blocks
        M, K, N, p = 3, 80, 2, 64
        ea = rng.integers(-5, 5, size=M * K)
        for k in range(40, 80):
            ea[np.arange(M) * K + k] += 900
        A = [random_balls(rng, M * K, 1, 64, exps=ea) for _ in "ri"]
        B = [random_balls(rng, K * N, 1, 64, -5, 5) for _ in "ri"]
        return A, B, M, K, N, p
    M, K, N, p = 4, 40, 3, 128
    A = [random_balls(rng, M * K, 2, 128, -20, 20) for _ in "ri"]
    B = [random_balls(rng, K * N, 2, 128, -20, 20) for _ in "ri"]
    if kind == "zero_im":
        A[1].flags[:] = X.FLAG_ZERO
        A[1].limbs[:] = 0
    return A, B, M, K, N, p


@pytest.mark.parametrize("kind", ["uniform", "structured", "zero_im", "banded"])
def test_complex_shared_blocks_reproduce_exact_product(kind):
    A, B, M, K, N, p = _complex_case(kind)
    blocks, re, im = recombined_complex(A, B, M, K, N, p)
    ere, eim = exact_complex_product(A, B, M, K, N)
    assert re == ere and im == eim
    assert blocks[0][0] == 0 and blocks[-1][1] == K
    if kind in ("uniform", "zero_im"):
        assert blocks == [(0, K, False)]
    if kind == "banded":
        assert blocks == [(0, 40, False), (40, 80, False)]


def test_eq2_equals_the_four_products_on_a_shared_block():
    A, B, M, K, N, p = _complex_case("uniform")
    e, f, Xs, Ys = alg2.scaled_block_complex(A, B, M, K, N, 0, K)
    R, I = alg2.eq2_block_products(Xs, Ys)
    mm = alg2.int_matmul
    rr, ii, ri, ir = mm(Xs[0], Ys[0]), mm(Xs[1], Ys[1]), mm(Xs[0], Ys[1]), mm(Xs[1], Ys[0])
    assert R == [[a - b for a, b in zip(x, y)] for x, y in zip(rr, ii)]
    assert I == [[a + b for a, b in zip(x, y)] for x, y in zip(ri, ir)]


def test_shared_scaling_is_minimal_over_both_parts():
    A, B, M, K, N, p = _complex_case("uniform")
    e, f, Xs, Ys = alg2.scaled_block_complex(A, B, M, K, N, 0, K)
    for i in range(M):
        assert any(v & 1 for q in (0, 1) for v in Xs[q][i])  # minimal over both parts
        for q in (0, 1):
            for k in range(K):
                assert Fraction(Xs[q][i][k]) == (ball_values(A[q], i * K + k)[0] *
                                                 Fraction(2) ** e[i])
    for j in range(N):
        assert any(Ys[q][k][j] & 1 for q in (0, 1) for k in range(K))


def test_planted_sign_slip_in_eq2_is_caught():
    def wrong(Xs, Ys):  # P3 = (X_re + X_im)(Y_re - Y_im)
        return alg2.eq2_block_products(Xs, (Ys[0], [[-v for v in r] for r in Ys[1]]))
    A, B, M, K, N, p = _complex_case("uniform")
    _, re, im = recombined_complex(A, B, M, K, N, p, products=wrong)
    ere, eim = exact_complex_product(A, B, M, K, N)
    assert (re, im) != (ere, eim)


# ------------------------------------------------------------------ complex, eq. 2 over shared blocks
# of the inner ordering (both suggestions of Sections IV-B and IV-C together)

def recombined_complex_ordered(A, B, M, K, N, prec, products=alg2.eq2_block_products):
    h, order, g, blocks = alg2.plan_complex_ordered(A, B, M, K, N, prec)
    re = [[Fraction(0)] * N for _ in range(M)]
    im = [[Fraction(0)] * N for _ in range(M)]
    for start, stop, base in blocks:
        ks = order[start:stop]
        if base:
            sub_re, sub_im = exact_complex_product(
                [_take(A[q], [i * K + k for i in range(M) for k in ks]) for q in (0, 1)],
                [_take(B[q], [k * N + j for k in ks for j in range(N)]) for q in (0, 1)],
                M, len(ks), N)
        else:
            e, f, Xs, Ys = alg2.scaled_block_complex_ordered(A, B, M, K, N, ks, g)
            R, I = products(Xs, Ys)
            sc = [[Fraction(2) ** (-e[i] - f[j]) for j in range(N)] for i in range(M)]
            sub_re = [[R[i][j] * sc[i][j] for j in range(N)] for i in range(M)]
            sub_im = [[I[i][j] * sc[i][j] for j in range(N)] for i in range(M)]
        for i in range(M):
            for j in range(N):
                re[i][j] += sub_re[i][j]
                im[i][j] += sub_im[i][j]
    return h, order, g, blocks, re, im


@pytest.mark.parametrize("kind", ["uniform", "structured", "zero_im", "banded"])
def test_complex_ordered_blocks_reproduce_exact_product(kind):
    A, B, M, K, N, p = _complex_case(kind)
    h, order, g, blocks, re, im = recombined_complex_ordered(A, B, M, K, N, p)
    ere, eim = exact_complex_product(A, B, M, K, N)
    assert re == ere and im == eim
    assert sorted(order) == list(range(K))
    assert blocks[0][0] == 0 and blocks[-1][1] == K
    if kind == "banded":  # products 2^895 apart cannot share a block, whatever the scaling
        assert blocks == [(0, 40, False), (40, 80, False)]
        assert sorted(order[:40]) == list(range(40))


def test_complex_ordering_merges_the_parts_tops():
    """a_k and b_k are the largest tops over both parts: the order and g agree with a direct
    computation from the merged columns and rows."""
    A, B, M, K, N, p = _complex_case("structured")
    order, g = alg2.inner_order_complex(A, B, M, K, N)
    keys = []
    for k in range(K):
        a = max(int(A[q].exp[i * K + k]) for q in (0, 1) for i in range(M)
                if not int(A[q].flags[i * K + k]) & X.FLAG_ZERO)
        b = max(int(B[q].exp[k * N + j]) for q in (0, 1) for j in range(N)
                if not int(B[q].flags[k * N + j]) & X.FLAG_ZERO)
        assert g[k] == math.floor((b - a) / 2)
        keys.append((a + b, k))
    assert order == [k for _, k in sorted(keys)]


def test_complex_ordering_leaves_full_blocks_on_a_structured_product():
    """The structured Laplace recipe at N = 128: the contiguous shared plan is all basecase, the
    shared plan over the merged order puts most indices in full blocks."""
    from synth.workloads import complex_matmul_laplace
    case = complex_matmul_laplace(n=128, structured=True)
    _, shared = alg2.plan_complex_shared(case.A, case.B, 128, 128, 128, 128)
    _, _, _, ordered = alg2.plan_complex_ordered(case.A, case.B, 128, 128, 128, 128)
    assert all(b for _, _, b in shared)
    assert sum(stop - start for start, stop, b in ordered if not b) >= 3 * 128 // 4


def test_complex_ordered_scaling_is_minimal_and_exact():
    A, B, M, K, N, p = _complex_case("structured")
    h, order, g, blocks = alg2.plan_complex_ordered(A, B, M, K, N, p)
    e, f, Xs, Ys = alg2.scaled_block_complex_ordered(A, B, M, K, N, order, g)
    for i in range(M):
        assert any(v & 1 for q in (0, 1) for v in Xs[q][i])
        for q in (0, 1):
            for t, k in enumerate(order):
                assert Fraction(Xs[q][i][t]) == (ball_values(A[q], i * K + k)[0] *
                                                 Fraction(2) ** (e[i] + g[k]))
    for j in range(N):
        assert any(Ys[q][t][j] & 1 for q in (0, 1) for t in range(K))
        for q in (0, 1):
            for t, k in enumerate(order):
                assert Fraction(Ys[q][t][j]) == (ball_values(B[q], k * N + j)[0] *
                                                 Fraction(2) ** (f[j] - g[k]))


def test_planted_mistakes_in_the_complex_ordering_are_caught(monkeypatch):
    # (a) the inner scaling applied to B with the wrong sign: the blocks no longer reproduce A B
    orig = alg2.scaled_block_complex_ordered

    def wrong_sign(A, B, M, K, N, ks, g):
        return orig(A, B, M, K, N, ks, [-v for v in g])
    A, B, M, K, N, p = _complex_case("structured")
    h, order, g, blocks = alg2.plan_complex_ordered(A, B, M, K, N, p)
    e, f, Xs, Ys = wrong_sign(A, B, M, K, N, order, g)
    bad = any(Fraction(Ys[0][t][j]) != ball_values(B[0], k * N + j)[0] * Fraction(2) ** (f[j] - g[k])
              for t, k in enumerate(order) for j in range(N))
    assert bad
    # (b) tops taken from the real part only: the order differs from the merged one
    only_re = alg2.inner_order(A[0], B[0], M, K, N)
    assert only_re != alg2.inner_order_complex(A, B, M, K, N)


# ------------------------------------------------------------------ negligible-limb omission
# (Section IV-B's last paragraph, in the reading of ``oracle.alg2.omission_thresholds``)

def _wide_case(seed, M, K, N, p, bits, spread):
    rng = np.random.default_rng(seed)
    nl = (bits + 63) // 64
    A = random_balls(rng, M * K, nl, bits, -spread, spread)
    B = random_balls(rng, K * N, nl, bits, -spread, spread)
    return A, B


@pytest.mark.parametrize("seed,M,K,N,p,bits,spread", [(1, 4, 12, 3, 64, 1024, 5),
                                                     (2, 5, 9, 4, 128, 200, 60),
                                                     (3, 3, 7, 6, 64, 64, 200)])
def test_omission_keeps_the_accuracy_bound(seed, M, K, N, p, bits, spread):
    """The truncated operands' exact product differs from the exact product by at most
    (3/64) 2^-p sum_k |a_ik b_kj| on every entry (the bound the reading derives), every dropped
    part of an entry is below 2^tau (2^sigma), and something is dropped at all."""
    from fractions import Fraction
    A, B = _wide_case(seed, M, K, N, p, bits, spread)
    tau, sigma = alg2.omission_thresholds(A, B, M, K, N, p)
    T = alg2.omitted_product(A, B, M, K, N, tau, sigma)
    S = exact_product(A, B, M, K, N)
    dropped = False
    for i in range(M):
        for k in range(K):
            tb = alg2.top_bottom(A, i * K + k)
            v, e = alg2.truncate_value(tb, tau[i])
            if tb is not None:
                exact = Fraction(tb[2]) * Fraction(2) ** tb[3]
                d = abs(exact - Fraction(v) * Fraction(2) ** e)
                assert d < Fraction(2) ** tau[i]
                dropped = dropped or d > 0
    for i in range(M):
        for j in range(N):
            sabs = sum(abs(ball_values(A, i * K + k)[0] * ball_values(B, k * N + j)[0])
                       for k in range(K))
            assert abs(T[i][j] - S[i][j]) <= Fraction(3, 64) * sabs / Fraction(2) ** p, (i, j)
    assert dropped


def test_omission_thresholds_by_brute_force():
    """tau_i and sigma_j against a direct evaluation of their definition (all pairs (i, j) and
    every k), on a case with zero entries and an empty row."""
    rng = np.random.default_rng(8)
    M, K, N, p = 4, 6, 5, 64
    A = random_balls(rng, M * K, 2, 128, -40, 40, zero_frac=0.3)
    B = random_balls(rng, K * N, 2, 128, -40, 40, zero_frac=0.3)
    A.flags[0:K] = X.FLAG_ZERO  # row 0 of A entirely zero: no product, no truncation
    A.limbs[:, 0:K] = 0
    tau, sigma = alg2.omission_thresholds(A, B, M, K, N, p)
    G = alg2.bc(K) + 8
    val = lambda raw, i: None if int(raw.flags[i]) & X.FLAG_ZERO else int(raw.exp[i])  # noqa
    for i in range(M):
        cand = []
        for j in range(N):
            prods = [val(A, i * K + k) + val(B, k * N + j) for k in range(K)
                     if val(A, i * K + k) is not None and val(B, k * N + j) is not None]
            cols = [val(B, k * N + j) for k in range(K) if val(B, k * N + j) is not None]
            if prods:
                cand.append(max(prods) - max(cols))
        assert tau[i] == (min(cand) - p - G if cand else None)
    assert tau[0] is None
    for j in range(N):
        cand = []
        for i in range(M):
            prods = [val(A, i * K + k) + val(B, k * N + j) for k in range(K)
                     if val(A, i * K + k) is not None and val(B, k * N + j) is not None]
            rows = [val(A, i * K + k) for k in range(K) if val(A, i * K + k) is not None]
            if prods:
                cand.append(max(prods) - max(rows))
        assert sigma[j] == (min(cand) - p - G if cand else None)


def test_planted_omission_slip_is_caught(monkeypatch):
    """Thresholds 150 bits higher than the reading's (as if E_ij were replaced by a bound 150
    bits too large) drop bits that matter: the accuracy pin fails."""
    orig = alg2.omission_thresholds

    def coarse(A, B, M, K, N, prec):
        tau, sigma = orig(A, B, M, K, N, prec)
        return ([None if t is None else t + 150 for t in tau],
                [None if t is None else t + 150 for t in sigma])
    monkeypatch.setattr(alg2, "omission_thresholds", coarse)
    with pytest.raises(AssertionError):
        test_omission_keeps_the_accuracy_bound(2, 5, 9, 4, 128, 200, 60)


# ------------------------------------------------------------------ omission for eq. 2
# (thresholds shared by both parts, in the reading of ``oracle.alg2.omission_thresholds_complex``)

# (A part, B part, sign) of the two products of each output part: Re, then Im
_PART_PRODUCTS = (((0, 0, 1), (1, 1, -1)), ((0, 1, 1), (1, 0, 1)))


def _complex_wide_case(seed, M, K, N, bits, spread, lopsided=False):
    """Complex operands with `bits`-bit mantissas; lopsided: A_re and B_im sit 2^200 lower than
    A_im and B_re, so every term of Re is about 2^-200 times the largest terms of Im."""
    rng = np.random.default_rng(seed)
    nl = (bits + 63) // 64
    lo = -200 if lopsided else 0
    A = [random_balls(rng, M * K, nl, bits, -spread + (lo if q == 0 else 0),
                      spread + (lo if q == 0 else 0)) for q in (0, 1)]
    B = [random_balls(rng, K * N, nl, bits, -spread + (lo if q == 1 else 0),
                      spread + (lo if q == 1 else 0)) for q in (0, 1)]
    return A, B


def _check_complex_omission(A, B, M, K, N, p, tau, sigma):
    """Each part of the truncated operands' product within (1/32) 2^-p sum |a b| of the exact part
    (the bound the reading derives); every dropped part below 2^tau (2^sigma); True when
    something was dropped."""
    re, im = alg2.omitted_product_complex(A, B, M, K, N, tau, sigma)
    ex = {(x, y): exact_product(A[x], B[y], M, K, N) for x in (0, 1) for y in (0, 1)}
    for part, got in enumerate((re, im)):
        for i in range(M):
            for j in range(N):
                S = sum(sg * ex[x, y][i][j] for x, y, sg in _PART_PRODUCTS[part])
                sabs = sum(abs(ball_values(A[x], i * K + k)[0] * ball_values(B[y], k * N + j)[0])
                           for x, y, _ in _PART_PRODUCTS[part] for k in range(K))
                assert abs(got[i][j] - S) <= Fraction(1, 32) * sabs / Fraction(2) ** p, \
                    (part, i, j)
    dropped = False
    for q in (0, 1):
        for i in range(M):
            for k in range(K):
                tb = alg2.top_bottom(A[q], i * K + k)
                if tb is None:
                    continue
                v, e = alg2.truncate_value(tb, tau[i])
                d = abs(Fraction(tb[2]) * Fraction(2) ** tb[3] - Fraction(v) * Fraction(2) ** e)
                assert tau[i] is not None or d == 0
                assert d == 0 or d < Fraction(2) ** tau[i]
                dropped = dropped or d > 0
    return dropped


@pytest.mark.parametrize("seed,M,K,N,p,bits,spread,lopsided", [
    (1, 4, 10, 3, 64, 512, 5, False), (2, 3, 8, 4, 128, 256, 60, False),
    (3, 3, 9, 3, 64, 320, 5, True)])
def test_complex_omission_keeps_the_accuracy_bound(seed, M, K, N, p, bits, spread, lopsided):
    A, B = _complex_wide_case(seed, M, K, N, bits, spread, lopsided)
    tau, sigma = alg2.omission_thresholds_complex(A, B, M, K, N, p)
    assert _check_complex_omission(A, B, M, K, N, p, tau, sigma)


def _thresholds_by_definition(A, B, M, K, N, p, larger_part_only=False):
    """tau_i and sigma_j evaluated directly from the exponent fields (2^(exp - 1) <= |x| < 2^exp):
    E per output part, or (larger_part_only) the larger of the two parts' E for both."""
    val = lambda raw, i: None if int(raw.flags[i]) & X.FLAG_ZERO else int(raw.exp[i])  # noqa
    G = alg2.bc(K) + 9

    def E(part, i, j):
        v = [val(A[x], i * K + k) + val(B[y], k * N + j) for x, y, _ in _PART_PRODUCTS[part]
             for k in range(K) if val(A[x], i * K + k) is not None
             and val(B[y], k * N + j) is not None]
        return max(v) if v else None

    def Es(i, j):
        e = [E(q, i, j) for q in (0, 1)]
        if larger_part_only:
            live = [v for v in e if v is not None]
            return [max(live)] if live else []
        return [v for v in e if v is not None]
    ctop = [max([val(B[q], k * N + j) for q in (0, 1) for k in range(K)
                 if val(B[q], k * N + j) is not None], default=None) for j in range(N)]
    rtop = [max([val(A[q], i * K + k) for q in (0, 1) for k in range(K)
                 if val(A[q], i * K + k) is not None], default=None) for i in range(M)]
    tau = []
    for i in range(M):
        cand = [e - ctop[j] for j in range(N) for e in Es(i, j)]
        tau.append(min(cand) - p - G if cand else None)
    sigma = []
    for j in range(N):
        cand = [e - rtop[i] for i in range(M) for e in Es(i, j)]
        sigma.append(min(cand) - p - G if cand else None)
    return tau, sigma


def test_complex_omission_thresholds_by_brute_force():
    """The shared thresholds against a direct evaluation of their definition, on a lopsided case
    with zero entries and a row of A that is zero in both parts."""
    rng = np.random.default_rng(9)
    M, K, N, p = 4, 6, 5, 64
    A = [random_balls(rng, M * K, 2, 128, -40 + (-90 if q == 0 else 0), 40, zero_frac=0.3)
         for q in (0, 1)]
    B = [random_balls(rng, K * N, 2, 128, -40, 40, zero_frac=0.3) for q in (0, 1)]
    for q in (0, 1):  # row 0 of A zero in both parts: no product, no truncation
        A[q].flags[0:K] = X.FLAG_ZERO
        A[q].limbs[:, 0:K] = 0
    tau, sigma = alg2.omission_thresholds_complex(A, B, M, K, N, p)
    assert (tau, sigma) == _thresholds_by_definition(A, B, M, K, N, p)
    assert tau[0] is None


def test_planted_complex_omission_slip_is_caught():
    """Thresholds taken from the larger part's bound for both parts (Im here) drop bits that
    matter to Re, about 2^-200 times smaller: the accuracy pin fails."""
    M, K, N, p = 3, 9, 3, 64
    A, B = _complex_wide_case(3, M, K, N, 320, 5, True)
    good = _thresholds_by_definition(A, B, M, K, N, p)
    assert good == alg2.omission_thresholds_complex(A, B, M, K, N, p)
    bad = _thresholds_by_definition(A, B, M, K, N, p, larger_part_only=True)
    with pytest.raises(AssertionError):
        _check_complex_omission(A, B, M, K, N, p, *bad)
