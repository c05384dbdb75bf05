"""The power series exponential (arbgpu_series_exp, Section V's dot-product recurrence) on the GPU
against the exact recurrence of ``oracle.series``: every output ball contains the exact
coefficient plus the radius that exact ball arithmetic would propagate, the closed form
exp(x) = sum x^k / k! is enclosed, and the radii stay within a modest factor of the precision."""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X
from oracle import series as S
from synth import random_balls
from tests.ballmake import make_balls
from tests.gpu_util import to_raw

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def _frac(dy):
    return X.dy_to_fraction(dy)


def _run(arb, A, length, batch, prec):
    ctx = arb.default_context()
    res = arb.Balls.empty(length * batch, (prec + 63) // 64)
    arb.series_exp(res, arb.Balls.from_raw(A), length, batch, prec, ctx=ctx)
    assert ctx.status() == 0
    return to_raw(res)


def _check(out, A, length, batch, prec, series_ids, loose_bits):
    worst = 0.0
    for s in series_ids:
        a = [_frac(X.mid(A, k * batch + s)) for k in range(length)]
        rho = [_frac(X.rad(A, k * batch + s)) for k in range(length)]
        b, r = S.exp_series_radius(a, rho, length)
        # the magnitude of the terms behind coefficient k: the exponential of |a|
        mag = S.exp_series([abs(v) for v in a], length)
        for k in range(length):
            m = _frac(X.mid(out, k * batch + s))
            rr = _frac(X.rad(out, k * batch + s))
            assert abs(m - b[k]) + r[k] <= rr, (s, k)
            worst = max(worst, float((rr - r[k]) / mag[k]))
    assert worst <= 2.0 ** (loose_bits - prec), worst
    return worst


@pytest.mark.parametrize("prec,length,rad", [(128, 40, None), (128, 32, 120), (256, 24, 250),
                                              (64, 50, None)])
def test_series_exp_contains_the_exact_coefficients(arb, prec, length, rad):
    rng = np.random.default_rng(prec + length)
    batch = 37
    nl = (prec + 63) // 64
    A = random_balls(rng, length * batch, nl, prec, -3, 1, rad_bits=rad, rad_zero_frac=0.3)
    out = _run(arb, A, length, batch, prec)
    _check(out, A, length, batch, prec, [0, 5, 17, 36], loose_bits=24)


def test_series_exp_of_x_encloses_inverse_factorials(arb):
    length, batch, prec = 60, 3, 128
    vals = []
    for k in range(length):
        for s in range(batch):
            vals.append(Fraction(1) if k == 1 else Fraction(0))
    A = make_balls(vals, nlimbs=2)
    out = _run(arb, A, length, batch, prec)
    for s in range(batch):
        for k in range(length):
            m = _frac(X.mid(out, k * batch + s))
            r = _frac(X.rad(out, k * batch + s))
            exact = Fraction(1, math.factorial(k))
            assert abs(m - exact) <= r, k
            assert r <= exact * Fraction(2) ** (16 - prec), k  # tight: a few ulps per step


def test_series_exp_argument_errors(arb):
    from paper_1901_04289_gb300 import _lib
    A = arb.Balls.empty(10, 2)
    with pytest.raises(_lib.ArbgpuError):
        arb.series_exp(arb.Balls.empty(10, 1), A, 5, 2, 128)  # output narrower than prec
    with pytest.raises(_lib.ArbgpuError):
        arb.series_exp(A, A, 5, 2, 128)  # aliasing


def test_series_graph_replay_matches_direct_launches(arb):
    """The recurrence's launches are recorded as a CUDA graph on the first call with given buffers
    and replayed by later identical calls: the replays write the same balls, bit for bit, as
    direct launches (ARBGPU_SERIES_GRAPH=0), and count the same kernels."""
    import contextlib

    from tests.gpu_util import env
    rng = np.random.default_rng(4242)
    prec, length, batch = 128, 30, 64
    A = random_balls(rng, length * batch, 2, 128, -3, 1, rad_bits=120, rad_zero_frac=0.5)
    ctx = arb.Context(0)
    a = arb.Balls.from_raw(A)
    res = arb.Balls.empty(length * batch, 2)
    outs, counts = [], []
    for mode in ("record", "replay", "direct"):
        for t in (res.limbs, res.exp, res.flags, res.rad_man, res.rad_exp):
            t.fill_(7)  # stale contents: each call must write every output
        n0 = ctx.launch_count()
        with (env(ARBGPU_SERIES_GRAPH="0") if mode == "direct" else contextlib.nullcontext()):
            arb.series_exp(res, a, length, batch, prec, ctx=ctx)
        assert ctx.status() == 0
        counts.append(ctx.launch_count() - n0)
        outs.append(to_raw(res))
    assert counts[0] == counts[1] == counts[2] > 2 * length
    for o in outs[1:]:
        for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
            assert np.array_equal(getattr(o, f), getattr(outs[0], f)), f
    _check(outs[0], A, length, batch, prec, range(0, batch, 9), 12)
