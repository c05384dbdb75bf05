"""Grouped batch (arbgpu_mat_mul_batched): every item matches what the single-product path gives
(the Algorithm 1 restatement bit for bit for classical items, containment and the accuracy bound for
block items), and all classical items run in one launch of the dot kernel."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import alg1
from oracle import exact as X
from synth import random_balls
from tests.gpu_util import mismatch, to_raw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def test_grouped_batch_mixed(arb):
    rng = np.random.default_rng(31)
    specs = [  # (n, p, complex)
        (16, 64, False), (23, 128, False), (40, 256, False), (17, 192, True), (29, 1024, False),
        (64, 128, False), (96, 256, False), (70, 128, True), (33, 512, False), (8, 2, False),
    ]
    items, raws = [], []
    for n, p, cplx in specs:
        nl = (p + 63) // 64
        parts = 2 if cplx else 1
        A = [random_balls(rng, n * n, nl, p, -30, 30, rad_bits=p - 8, rad_zero_frac=0.5)
             for _ in range(parts)]
        B = [random_balls(rng, n * n, nl, p, -30, 30, rad_bits=p - 8, rad_zero_frac=0.5)
             for _ in range(parts)]
        C = [arb.Balls.empty(n * n, nl) for _ in range(parts)]
        dA = [arb.Balls.from_raw(a) for a in A]
        dB = [arb.Balls.from_raw(b) for b in B]
        items.append(dict(C=C if cplx else C[0], A=dA if cplx else dA[0],
                          B=dB if cplx else dB[0], M=n, K=n, N=n, prec=p))
        raws.append((A, B, C, n, p, cplx))
    ctx = arb.default_context()
    ctx.trace(True)
    arb.mat_mul_batched(items)
    assert ctx.status() == 0
    names = [r[0] for r in ctx.trace_read()]
    ctx.trace(False)
    assert names.count("dot_setup") == 1  # every classical item in one grouped launch
    rng2 = np.random.default_rng(2)
    for A, B, C, n, p, cplx in raws:
        outs = [to_raw(c) for c in C]
        nl = (p + 63) // 64
        for _ in range(12):
            i, j = int(rng2.integers(n)), int(rng2.integers(n))
            idx = i * n + j
            xi = [i * n + k for k in range(n)]
            yi = [k * n + j for k in range(n)]
            if n < 48:  # classical item: bit for bit
                if cplx:
                    re, im = alg1.complex_dot_raw(A, xi, B, yi, p, nl)
                    assert mismatch(outs[0], idx, re) is None
                    assert mismatch(outs[1], idx, im) is None
                else:
                    assert mismatch(outs[0], idx, alg1.dot_raw(A[0], xi, B[0], yi, p, nl)) is None
            else:  # block item: containment and accuracy
                if cplx:
                    terms = X.complex_dot_terms(A, xi, B, yi)
                else:
                    terms = (X.real_dot_terms(A[0], xi, B[0], yi),)
                for part, t in enumerate(terms):
                    S, Sabs, R = X.dot_terms_exact(t)
                    m, r = X.mid(outs[part], idx), X.rad(outs[part], idx)
                    assert X.contains(m, r, S, R)
                    assert X.accuracy_ratio(m, S, Sabs, p) <= 1.0


def test_grouped_batch_complex_3m_matches_single_calls(arb):
    """Complex block items with ARBGPU_MM_COMPLEX_3M in a grouped batch give, field for field, what
    the single-product call with the same flag gives (eq. 2, Section IV-C), next to a real item."""
    rng = np.random.default_rng(32)
    specs = [(64, 128, True), (80, 256, False), (72, 192, True)]
    items, singles, outs = [], [], []
    for n, p, cplx in specs:
        nl = (p + 63) // 64
        parts = 2 if cplx else 1
        A = [arb.Balls.from_raw(random_balls(rng, n * n, nl, p, -10, 10, rad_bits=p - 8,
                                             rad_zero_frac=0.5)) for _ in range(parts)]
        B = [arb.Balls.from_raw(random_balls(rng, n * n, nl, p, -10, 10, rad_bits=p - 8,
                                             rad_zero_frac=0.5)) for _ in range(parts)]
        Cb = [arb.Balls.empty(n * n, nl) for _ in range(parts)]
        Cs = [arb.Balls.empty(n * n, nl) for _ in range(parts)]
        pick = (lambda v: v) if cplx else (lambda v: v[0])
        items.append(dict(C=pick(Cb), A=pick(A), B=pick(B), M=n, K=n, N=n, prec=p,
                          alg=arb.ALG_BLOCK, flags=arb.MM_COMPLEX_3M))
        arb.mat_mul(pick(Cs), pick(A), pick(B), n, n, n, p, alg=arb.ALG_BLOCK,
                    flags=arb.MM_COMPLEX_3M)
        outs.append(Cb)
        singles.append(Cs)
    ctx = arb.default_context()
    ctx.trace(True)
    arb.mat_mul_batched(items)
    assert ctx.status() == 0
    names = [r[0] for r in ctx.trace_read()]
    ctx.trace(False)
    assert names.count("z3m") == 2  # both complex items took eq. 2
    for Cb, Cs in zip(outs, singles):
        for a, b in zip(Cb, Cs):
            ra, rb = to_raw(a), to_raw(b)
            for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
                assert np.array_equal(getattr(ra, f), getattr(rb, f)), f
