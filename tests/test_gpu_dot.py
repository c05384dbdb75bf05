"""Kernel (a) on the GPU against the Algorithm 1 restatement (bit for bit) and the exact oracle
(containment, accuracy), through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import alg1
from oracle import exact as X
from synth import FLAG_NAN, RawBalls, SEED_BASE, random_balls
from synth.workloads import DotBatch, batched_dots, dot_matmul_n32_p128, matmul_uniform
from tests.gpu_util import batch_tensors, mismatch, to_raw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def run_batch(arb, batch: DotBatch, nl_out=None, complex_parts=None, approx=False,
              reduce_prec=False):
    import torch
    nl_out = nl_out or (int(batch.prec.max()) + 63) // 64
    n = int(batch.length.shape[0])
    x = arb.Balls.from_raw(batch.x)
    y = arb.Balls.from_raw(batch.y)
    res = arb.Balls.empty(n, nl_out)
    init = arb.Balls.from_raw(batch.initial) if batch.initial is not None else None
    t = batch_tensors(batch)
    arb.dot(res, x, y, t["xoff"], t["xstep"], t["yoff"], t["ystep"], t["length"], t["prec"],
            prec_max=int(batch.prec.max()), len_max=int(batch.length.max()), sub=t["sub"],
            initial=init, approx=approx, reduce_prec=reduce_prec)
    st = arb.default_context().status()
    torch.cuda.synchronize()
    return to_raw(res), st


def alg1_of(batch: DotBatch, b: int, nl_out: int, reduce_prec=False):
    idx_x = [int(batch.xoff[b] + i * batch.xstep[b]) for i in range(int(batch.length[b]))]
    idx_y = [int(batch.yoff[b] + i * batch.ystep[b]) for i in range(int(batch.length[b]))]
    init = (batch.initial, b) if batch.initial is not None else None
    return alg1.dot_raw(batch.x, idx_x, batch.y, idx_y, int(batch.prec[b]), nl_out,
                        sub=bool(batch.sub[b]), initial=init, reduce_prec=reduce_prec)


def small_batch(seed, count, nl, precs, spread, rad_bits, rad_zero, zero_frac=0.0, lmax=70,
                with_init=False, strides=False):
    rng = np.random.default_rng(seed)
    length = rng.integers(0, lmax, size=count, endpoint=True).astype(np.int64)
    prec = rng.choice(np.asarray(precs, dtype=np.int32), size=count).astype(np.int32)
    total = int(length.sum()) + 1
    mb = rng.integers(1, 64 * nl + 1, size=total)
    x = random_balls(rng, total, nl, mb, -spread, spread, rad_bits=rad_bits,
                     rad_zero_frac=rad_zero, zero_frac=zero_frac)
    y = random_balls(rng, total, nl, rng.permutation(mb), -spread, spread, rad_bits=rad_bits,
                     rad_zero_frac=rad_zero, zero_frac=zero_frac)
    off = np.zeros(count, dtype=np.int64)
    off[1:] = np.cumsum(length)[:-1]
    xstep = np.ones(count, dtype=np.int64)
    ystep = np.ones(count, dtype=np.int64)
    xoff, yoff = off.copy(), off.copy()
    if strides:  # reverse every other dot (negative stride) and read y from a shifted window
        rev = (np.arange(count) % 2) == 1
        xoff[rev] = off[rev] + np.maximum(length[rev] - 1, 0)
        xstep[rev] = -1
        ystep[::3] = 0  # a zero stride repeats one entry
    sub = rng.integers(0, 2, size=count).astype(np.uint8)
    init = random_balls(rng, count, nl, 64 * nl, -spread, spread, rad_bits=rad_bits,
                        rad_zero_frac=rad_zero, zero_frac=zero_frac) if with_init else None
    return DotBatch("small", x, y, xoff, xstep, yoff, ystep, length, prec, sub, init)


SMALL = [
    dict(seed=1, count=300, nl=1, precs=(2, 3, 53, 64), spread=10, rad_bits=None, rad_zero=0),
    dict(seed=2, count=300, nl=2, precs=(64, 100, 128), spread=40, rad_bits=100, rad_zero=0.5,
         zero_frac=0.1, with_init=True),
    dict(seed=3, count=200, nl=3, precs=(65, 128, 192), spread=300, rad_bits=150, rad_zero=0.3,
         strides=True),
    dict(seed=4, count=100, nl=4, precs=(200, 256), spread=20, rad_bits=250, rad_zero=0.0,
         with_init=True, strides=True),
    dict(seed=5, count=60, nl=8, precs=(300, 512), spread=600, rad_bits=400, rad_zero=0.5,
         zero_frac=0.2),
    dict(seed=6, count=40, nl=16, precs=(700, 1024), spread=2000, rad_bits=900, rad_zero=0.5,
         lmax=40, with_init=True),
    dict(seed=7, count=50, nl=3, precs=(64,), spread=5, rad_bits=None, rad_zero=0, lmax=300),
]


@pytest.mark.parametrize("k", range(len(SMALL)))
def test_batched_dots_bit_exact_vs_alg1(arb, k):
    batch = small_batch(**SMALL[k])
    nl_out = (int(batch.prec.max()) + 63) // 64
    out, st = run_batch(arb, batch, nl_out)
    assert st == 0
    bad = []
    for b in range(len(batch.length)):
        ref = alg1_of(batch, b, nl_out)
        mm = mismatch(out, b, ref)
        if mm:
            bad.append((b, mm))
    assert not bad, f"{len(bad)} mismatches, first: {bad[:2]}"


@pytest.mark.parametrize("k", [0, 1, 2, 6])
def test_fused_launch_agrees_with_class_launches(arb, k):
    """Batches whose largest size class is small run setup and evaluation in one fused launch;
    the setup launch plus one launch per class (ARBGPU_DOT_FUSED=0) gives the same balls, bit for
    bit, and the same status."""
    from tests.gpu_util import env
    batch = small_batch(**SMALL[k])
    nl_out = (int(batch.prec.max()) + 63) // 64
    fused, st1 = run_batch(arb, batch, nl_out)
    with env(ARBGPU_DOT_FUSED="0"):
        split, st2 = run_batch(arb, batch, nl_out)
    assert st1 == st2 == 0
    for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
        assert np.array_equal(getattr(fused, f), getattr(split, f)), f


@pytest.mark.parametrize("k", [1, 2, 4, 5])
def test_reduced_precision_dots_bit_exact_vs_alg1(arb, k):
    """ARBGPU_DOT_REDUCE_PREC (Section III-C, "optimize p"): every output field equals the Algorithm 1
    restatement run with the same reduction, and the reduction changes some results."""
    batch = small_batch(**SMALL[k])
    nl_out = (int(batch.prec.max()) + 63) // 64
    out, st = run_batch(arb, batch, nl_out, reduce_prec=True)
    full, _ = run_batch(arb, batch, nl_out)
    assert st == 0
    bad = []
    for b in range(len(batch.length)):
        mm = mismatch(out, b, alg1_of(batch, b, nl_out, reduce_prec=True))
        if mm:
            bad.append((b, mm))
    assert not bad, f"{len(bad)} mismatches, first: {bad[:2]}"
    assert not (np.array_equal(out.limbs, full.limbs) and np.array_equal(out.rad_man,
                                                                          full.rad_man))


@pytest.mark.parametrize("k", [1, 2, 4, 5])
def test_approx_dots_give_the_ball_midpoints(arb, k):
    """arbgpu_approx_dot (midpoints only, the approx_dot interface of Section III): every midpoint
    is the one arbgpu_dot gives (the same accumulation and rounding), bit for bit, whatever the
    radii; every output radius is zero."""
    batch = small_batch(**SMALL[k])
    nl_out = (int(batch.prec.max()) + 63) // 64
    ball, st = run_batch(arb, batch, nl_out)
    appr, st2 = run_batch(arb, batch, nl_out, approx=True)
    assert st == 0 and st2 == 0
    assert np.array_equal(ball.limbs, appr.limbs)
    assert np.array_equal(ball.exp, appr.exp)
    assert np.array_equal(ball.flags, appr.flags)
    assert not np.any(appr.rad_man) and not np.any(appr.rad_exp)
    assert np.any(ball.rad_man)  # the ball dots had radii to ignore


@pytest.mark.parametrize("k", [1, 2, 4])
def test_batched_dots_contain_exact(arb, k):
    batch = small_batch(**SMALL[k])
    nl_out = (int(batch.prec.max()) + 63) // 64
    out, _ = run_batch(arb, batch, nl_out)
    for b in range(0, len(batch.length), 3):
        idx_x = [int(batch.xoff[b] + i * batch.xstep[b]) for i in range(int(batch.length[b]))]
        idx_y = [int(batch.yoff[b] + i * batch.ystep[b]) for i in range(int(batch.length[b]))]
        terms = X.real_dot_terms(batch.x, idx_x, batch.y, idx_y, bool(batch.sub[b]))
        init = X.ball(batch.initial, b) if batch.initial is not None else None
        S, Sabs, R = X.dot_terms_exact(terms, init)
        m, r = X.mid(out, b), X.rad(out, b)
        assert X.contains(m, r, S, R)


def test_config_matmul_n32_p128_by_dots(arb):
    import torch
    case = dot_matmul_n32_p128()
    A, B = arb.Balls.from_raw(case.A[0]), arb.Balls.from_raw(case.B[0])
    Cd = arb.Balls.empty(32 * 32, 2)
    arb.mat_mul(Cd, A, B, 32, 32, 32, 128, alg=arb.ALG_DOT)
    assert arb.default_context().status() == 0
    out = to_raw(Cd)
    worst = 0.0
    for i in range(32):
        for j in range(32):
            ref = alg1.matmul_entry(case.A[0], case.B[0], 32, 32, i, j, 128, 2)
            assert mismatch(out, i * 32 + j, ref) is None
            S, Sabs, R = X.dot_terms_exact(X.matmul_entry_terms(case.A[0], case.B[0], 32, 32, i, j))
            m, r = X.mid(out, i * 32 + j), X.rad(out, i * 32 + j)
            assert X.contains(m, r, S, R)
            worst = max(worst, X.accuracy_ratio(m, S, Sabs, 128))
    assert worst <= 1.0
    torch.cuda.synchronize()


def test_full_batched_dots_sampled(arb):
    batch = batched_dots()
    out, st = run_batch(arb, batch, 3)
    assert st == 0
    rng = np.random.default_rng(0)
    sample = rng.choice(len(batch.length), size=600, replace=False)
    worst = 0.0
    for b in sample:
        ref = alg1_of(batch, int(b), 3)
        assert mismatch(out, int(b), ref) is None, int(b)
        idx = range(int(batch.xoff[b]), int(batch.xoff[b] + batch.length[b]))
        S, Sabs, R = X.dot_terms_exact(X.real_dot_terms(batch.x, idx, batch.y, idx))
        m, r = X.mid(out, int(b)), X.rad(out, int(b))
        assert X.contains(m, r, S, R)
        worst = max(worst, X.accuracy_ratio(m, S, Sabs, int(batch.prec[b])))
    assert worst <= 1.0
    # every output is a finite ball in the expected format
    assert not (out.flags & FLAG_NAN).any()


def test_complex_dots_vs_alg1(arb):
    import torch
    rng = np.random.default_rng(11)
    n, L, nl, p = 40, 25, 2, 128
    tot = n * L
    xs = [random_balls(rng, tot, nl, 128, -30, 30, rad_bits=120, rad_zero_frac=0.5) for _ in (0, 1)]
    ys = [random_balls(rng, tot, nl, 128, -30, 30, rad_bits=120, rad_zero_frac=0.5) for _ in (0, 1)]
    ini = [random_balls(rng, n, nl, 128, -30, 30, rad_bits=120) for _ in (0, 1)]
    off = np.arange(n, dtype=np.int64) * L
    dev = lambda a, dt: torch.as_tensor(a, dtype=dt, device="cuda")  # noqa
    xb = [arb.Balls.from_raw(v) for v in xs]
    yb = [arb.Balls.from_raw(v) for v in ys]
    ib = [arb.Balls.from_raw(v) for v in ini]
    res = [arb.Balls.empty(n, nl), arb.Balls.empty(n, nl)]
    sub = (np.arange(n) % 2).astype(np.uint8)
    arb.dot(res, xb, yb, dev(off, torch.int64), dev(np.ones(n), torch.int64), dev(off, torch.int64),
            dev(np.ones(n), torch.int64), dev(np.full(n, L), torch.int64),
            dev(np.full(n, p), torch.int32), prec_max=p, len_max=L, sub=dev(sub, torch.uint8),
            initial=ib)
    assert arb.default_context().status() == 0
    outs = [to_raw(r) for r in res]
    for b in range(n):
        idx = list(range(b * L, (b + 1) * L))
        re, im = alg1.complex_dot_raw(xs, idx, ys, idx, p, nl, sub=bool(sub[b]),
                                      initial=((ini[0], ini[1]), b))
        assert mismatch(outs[0], b, re) is None
        assert mismatch(outs[1], b, im) is None


def test_edge_cases(arb):
    """Empty dots, all-zero inputs, exact cancellation, special values, huge exponents."""
    import torch
    rng = np.random.default_rng(5)
    x = random_balls(rng, 12, 2, 128, -5, 5, rad_bits=100)
    y = random_balls(rng, 12, 2, 128, -5, 5)
    # dot 0: empty; dot 1: zeros; dot 2: x*1 - x*1; dot 3: NaN; dot 4: exponent 2^60; dot 5: ok
    for i in (2, 3):
        x.flags[i] = X.FLAG_ZERO
        x.limbs[:, i] = 0
    y.limbs[:, 4] = 0
    y.limbs[1, 4] = np.uint64(1 << 63)
    y.exp[4] = 1
    y.flags[4] = 1 << 8
    y.limbs[:, 5] = y.limbs[:, 4]
    y.exp[5] = 1
    y.flags[5] = (1 << 8) | 1
    x.limbs[:, 5] = x.limbs[:, 4]
    x.exp[5] = x.exp[4]
    x.flags[5] = x.flags[4]
    x.rad_man[4:6] = 0
    x.rad_exp[4:6] = 0
    x.flags[6] = FLAG_NAN
    x.exp[8] = 1 << 60
    xoff = np.array([0, 2, 4, 6, 8, 10], dtype=np.int64)
    length = np.array([0, 2, 2, 1, 1, 2], dtype=np.int64)
    batch = DotBatch("edge", x, y, xoff, np.ones(6, np.int64), xoff.copy(), np.ones(6, np.int64),
                     length, np.full(6, 128, np.int32), np.zeros(6, np.uint8))
    out, st = run_batch(arb, batch, 2)
    assert st == 2  # ARBGPU_ERR_UNSUPPORTED_VALUE
    for b in range(6):
        assert mismatch(out, b, alg1_of(batch, b, 2)) is None, b
    assert out.flags[0] == X.FLAG_ZERO and out.rad_man[0] == 0
    assert out.flags[2] == X.FLAG_ZERO and out.rad_man[2] == 0  # x - x = [0 +- 0]
    assert out.flags[3] & FLAG_NAN and out.flags[4] & FLAG_NAN
    torch.cuda.synchronize()


def test_rejects_bad_arguments(arb):
    import torch
    batch = small_batch(**SMALL[0])
    x = arb.Balls.from_raw(batch.x)
    res = arb.Balls.empty(len(batch.length), 1)
    t = batch_tensors(batch)
    with pytest.raises(arb.ArbgpuError):  # output aliasing an input
        arb.dot(x, x, x, t["xoff"], t["xstep"], t["yoff"], t["ystep"], t["length"], t["prec"],
                prec_max=64, len_max=int(batch.length.max()))
    with pytest.raises(arb.ArbgpuError):  # precision beyond the output's limbs
        arb.dot(res, x, x, t["xoff"], t["xstep"], t["yoff"], t["ystep"], t["length"], t["prec"],
                prec_max=200, len_max=int(batch.length.max()))
    # a dot longer than the stated len_max is flagged on the device
    arb.dot(res, x, x, t["xoff"], t["xstep"], t["yoff"], t["ystep"], t["length"], t["prec"],
            prec_max=64, len_max=1)
    assert arb.default_context().status() == 6
    torch.cuda.synchronize()


def test_matmul_by_dots_p256_sampled(arb):
    case = matmul_uniform(SEED_BASE + 3, 96, 256, -20, 20, rad_bits=250)
    A, B = arb.Balls.from_raw(case.A[0]), arb.Balls.from_raw(case.B[0])
    Cd = arb.Balls.empty(96 * 96, 4)
    arb.mat_mul(Cd, A, B, 96, 96, 96, 256, alg=arb.ALG_DOT)
    assert arb.default_context().status() == 0
    out = to_raw(Cd)
    rng = np.random.default_rng(1)
    for e in rng.choice(96 * 96, 150, replace=False):
        i, j = divmod(int(e), 96)
        ref = alg1.matmul_entry(case.A[0], case.B[0], 96, 96, i, j, 256, 4)
        assert mismatch(out, int(e), ref) is None


@pytest.mark.parametrize("M,K,N,prec,cplx", [(330, 70, 450, 128, False), (200, 129, 400, 256, False),
                                             (90, 40, 700, 512, False), (200, 33, 360, 1024, False),
                                             (310, 50, 330, 64, True), (400, 17, 130, 192, True)])
def test_tiled_matrix_dots_equal_the_lane_group_kernel(arb, M, K, N, prec, cplx):
    """The classical product through the shared-memory tiled dot kernel equals, in every output
    field, the group-of-lanes kernel (ARBGPU_DOT_TILE=0) and the Algorithm 1 restatement."""
    import os

    from tests.gpu_util import to_raw
    rng = np.random.default_rng(M * 1000 + K)
    nl = (prec + 63) // 64
    parts = 2 if cplx else 1
    A = [random_balls(rng, M * K, nl, prec, -12, 12, rad_bits=prec - 6, rad_zero_frac=0.4,
                      zero_frac=0.1) for _ in range(parts)]
    B = [random_balls(rng, K * N, nl, prec, -12, 12, rad_bits=prec - 6, rad_zero_frac=0.4,
                      zero_frac=0.1) for _ in range(parts)]
    outs = []
    for tile in ("1", "0"):
        old = os.environ.get("ARBGPU_DOT_TILE")
        os.environ["ARBGPU_DOT_TILE"] = tile
        try:
            C = [arb.Balls.empty(M * N, nl) for _ in range(parts)]
            ctx = arb.default_context()
            ctx.trace(True)
            arb.mat_mul(C if cplx else C[0], [arb.Balls.from_raw(a) for a in A] if cplx
                        else arb.Balls.from_raw(A[0]), [arb.Balls.from_raw(b) for b in B] if cplx
                        else arb.Balls.from_raw(B[0]), M, K, N, prec, alg=arb.ALG_DOT)
            assert ctx.status() == 0
            names = [r[0] for r in ctx.trace_read()]
            ctx.trace(False)
            assert ("dot_tile" in names) == (tile == "1")
            outs.append([to_raw(c) for c in C])
        finally:
            if old is None:
                del os.environ["ARBGPU_DOT_TILE"]
            else:
                os.environ["ARBGPU_DOT_TILE"] = old
    for a, b in zip(outs[0], outs[1]):
        for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
    if not cplx:
        for e in range(0, M * N, 997):
            i, j = divmod(e, N)
            ref = alg1.matmul_entry(A[0], B[0], K, N, i, j, prec, nl)
            assert mismatch(outs[0][0], e, ref) is None, (i, j)
