"""The autotuner (arbgpu_set_autotune).  Engines: the first block product of a size bucket runs on
both integer engines and keeps the faster, later products of the bucket reuse that choice, and the
balls are bit-identical to those of the untuned call (the two engines give the same exact integer
products, Section IV-A), which are the exactly rounded values of the exact products.  Algorithms:
ALG_AUTO products near the dot / block crossover (Section V) are timed once per size bucket, and
their balls are those of the chosen algorithm."""
from __future__ import annotations

import numpy as np
import pytest

from synth import random_balls
from tests.gpu_util import env, to_raw
from tests.test_gpu_block import check_bounds, check_entries

pytestmark = pytest.mark.gpu


def _mm(arb, ctx, A, B, M, K, N, p):
    C = arb.Balls.empty(M * N, (p + 63) // 64)
    arb.mat_mul(C, arb.Balls.from_raw(A), arb.Balls.from_raw(B), M, K, N, p, alg=arb.ALG_BLOCK,
                ctx=ctx)
    assert ctx.status() == 0
    return to_raw(C)


def _same(a, b):
    return all(np.array_equal(getattr(a, f), getattr(b, f))
               for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"))


def test_autotune_picks_once_per_bucket_and_keeps_the_results():
    import paper_1901_04289_gb300 as arb
    rng = np.random.default_rng(77)
    cases = [(96, 96, 96, 128, 20, 2), (80, 64, 72, 256, 30, 4)]
    data = []
    for M, K, N, p, spread, nl in cases:
        A = random_balls(rng, M * K, nl, 64 * nl, -spread, spread, rad_bits=p - 8,
                         rad_zero_frac=0.5)
        B = random_balls(rng, K * N, nl, 64 * nl, -spread, spread, rad_bits=p - 8,
                         rad_zero_frac=0.5)
        data.append((A, B, M, K, N, p))
    with env(ARBGPU_OMIT="0"):
        plain = arb.Context(0)  # tuner off (the default)
        refs = [_mm(arb, plain, *d) for d in data]
        assert plain.autotune_stats() == dict(buckets=0, timing_runs=0, crt_buckets=0)
        tuned = arb.Context(0)
        tuned.set_autotune(True)
        for q, d in enumerate(data):
            out = _mm(arb, tuned, *d)
            st = tuned.autotune_stats()
            # one new bucket, decided by running both engines twice each (untimed, then timed)
            assert st["buckets"] == q + 1 and st["timing_runs"] == 4 * (q + 1), st
            assert _same(out, refs[q])
            # the decided bucket: no more timing runs, the same balls
            n0 = tuned.launch_count()
            again = _mm(arb, tuned, *d)
            assert tuned.autotune_stats() == st
            assert _same(again, refs[q])
            # the repeat launched one product's kernels, not two engines' worth
            n_plain0 = plain.launch_count()
            _mm(arb, plain, *d)
            assert tuned.launch_count() - n0 <= plain.launch_count() - n_plain0 + 2
        for (A, B, M, K, N, p), ref in zip(data, refs):
            rng2 = np.random.default_rng(M + N)
            ents = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 6), rng2.integers(0, N, 6))]
            check_entries(ref, A, B, M, K, N, p, ents, (p + 63) // 64)


def _mm_alg(arb, ctx, A, B, M, K, N, p, alg):
    C = arb.Balls.empty(M * N, (p + 63) // 64)
    arb.mat_mul(C, arb.Balls.from_raw(A), arb.Balls.from_raw(B), M, K, N, p, alg=alg, ctx=ctx)
    assert ctx.status() == 0
    return to_raw(C)


AUTO_CASES = [(40, 64, 40, 128, 10, 2), (96, 128, 80, 256, 20, 4), (64, 64, 64, 1024, 30, 16)]


def test_auto_algorithm_is_timed_once_per_bucket():
    """ALG_AUTO near the dot / block crossover with the autotuner on: the first product of a size
    bucket runs both algorithms (twice each) and keeps the faster; its balls are, bit for bit,
    those of the chosen algorithm run explicitly, and a second product of the bucket runs no
    timing and gives the same balls.  Every sampled ball contains the exact product."""
    import paper_1901_04289_gb300 as arb
    rng = np.random.default_rng(91)
    plain = arb.Context(0)
    tuned = arb.Context(0)
    tuned.set_autotune(True)
    for q, (M, K, N, p, spread, nl) in enumerate(AUTO_CASES):
        A = random_balls(rng, M * K, nl, 64 * nl, -spread, spread, rad_bits=p - 8,
                         rad_zero_frac=0.5)
        B = random_balls(rng, K * N, nl, 64 * nl, -spread, spread, rad_bits=p - 8,
                         rad_zero_frac=0.5)
        ref = {alg: _mm_alg(arb, plain, A, B, M, K, N, p, alg)
               for alg in (arb.ALG_DOT, arb.ALG_BLOCK)}
        before = tuned.autotune_alg_stats()
        out = _mm_alg(arb, tuned, A, B, M, K, N, p, arb.ALG_AUTO)
        st = tuned.autotune_alg_stats()
        assert st["buckets"] == q + 1 and st["timing_runs"] == before["timing_runs"] + 4, st
        chose_block = st["block_buckets"] > before["block_buckets"]
        want = ref[arb.ALG_BLOCK if chose_block else arb.ALG_DOT]
        assert _same(out, want), (M, K, N, p, chose_block)
        again = _mm_alg(arb, tuned, A, B, M, K, N, p, arb.ALG_AUTO)
        assert tuned.autotune_alg_stats() == st
        assert _same(again, want)
        rng2 = np.random.default_rng(M + p)
        ents = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 5), rng2.integers(0, N, 5))]
        check_bounds(out, A, B, M, K, N, p, ents)


def test_batched_auto_items_are_timed_before_the_batch():
    """In a batched call with the autotuner on, AUTO items of undecided buckets are timed alone
    first; the batch then runs each with its bucket's choice, so every item's balls equal those
    of the chosen algorithm, and a repeated batch times nothing."""
    import paper_1901_04289_gb300 as arb
    rng = np.random.default_rng(92)
    plain = arb.Context(0)
    tuned = arb.Context(0)
    tuned.set_autotune(True)
    data = []
    for M, K, N, p, spread, nl in AUTO_CASES[:2] + [(32, 32, 32, 128, 10, 2)]:
        A = random_balls(rng, M * K, nl, 64 * nl, -spread, spread, rad_bits=p - 8)
        B = random_balls(rng, K * N, nl, 64 * nl, -spread, spread, rad_bits=p - 8)
        data.append((A, B, M, K, N, p))

    def batch():
        items = [dict(C=arb.Balls.empty(M * N, (p + 63) // 64), A=arb.Balls.from_raw(A),
                      B=arb.Balls.from_raw(B), M=M, K=K, N=N, prec=p)
                 for A, B, M, K, N, p in data]
        arb.mat_mul_batched(items, ctx=tuned)
        assert tuned.status() == 0
        return [to_raw(it["C"]) for it in items]
    outs = batch()
    st = tuned.autotune_alg_stats()
    assert st["buckets"] == len(data)
    again = batch()
    assert tuned.autotune_alg_stats() == st
    for (A, B, M, K, N, p), o1, o2 in zip(data, outs, again):
        refs = [_mm_alg(arb, plain, A, B, M, K, N, p, alg) for alg in (arb.ALG_DOT, arb.ALG_BLOCK)]
        assert _same(o1, o2)
        assert any(_same(o1, r) for r in refs), (M, K, N, p)
