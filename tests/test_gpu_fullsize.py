"""Parity on sampled entries of the full-size workloads the bench times, through the C ABI:

* the complex N = 2048, p = 128 product with Laplace(40) exponents, both the structured variant
  (exponent blocks along the inner index) and the literal one (i.i.d. exponents): containment of
  the exact product and the accuracy bound |m - S| <= 2^-p sum |a b| on every sampled entry, by
  four real products with their negligible limbs omitted, with ARBGPU_MM_COMPLEX_3M by eq. 2 on
  both parts truncated under shared thresholds, and with the omission off by eq. 2 over several
  blocks shared by both parts (over their shared inner order);
* the grouped batch of 256 real products (N in [16, 512], p in {64, ..., 1024}) in one
  arbgpu_mat_mul_batched call: block items (one exponent block each) bit-exact RNE_p of the exact
  sum, or within the bound where negligible limbs were omitted, classical items bit-exact against
  the Algorithm 1 restatement, containment everywhere, including the p = 1024 items whose
  reconstruction runs on the CUDA cores."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import alg1
from oracle import exact as X
from synth.workloads import complex_matmul_laplace, grouped_matmuls
from tests.gpu_util import entry_fields, expected_fields, to_raw
from tests.test_gpu_block import check_bounds, check_complex, check_entries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


@pytest.mark.parametrize("structured", [True, False])
@pytest.mark.parametrize("mode", ["4m", "3m", "3m_several"])
def test_complex2048_sampled(arb, structured, mode):
    from tests.gpu_util import env
    case = complex_matmul_laplace(structured=structured)
    n, p = case.N, case.prec
    A = [arb.Balls.from_raw(a) for a in case.A]
    B = [arb.Balls.from_raw(b) for b in case.B]
    C = [arb.Balls.empty(n * n, 2), arb.Balls.empty(n * n, 2)]
    flags = 0 if mode == "4m" else arb.MM_COMPLEX_3M
    need = arb.mat_mul_workspace_size(n, n, n, p, 2, 2, True, arb.ALG_AUTO, flags)
    import torch
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    ctx = arb.default_context()
    # 3m_several: the omission off, so eq. 2 runs over several blocks shared by both parts
    import contextlib
    with env(ARBGPU_OMIT="0") if mode == "3m_several" else contextlib.nullcontext():
        arb.mat_mul(C, A, B, n, n, n, p, flags=flags, workspace=ws, ctx=ctx)
    assert ctx.status() == 0
    plans = ctx.last_plans()
    if mode == "3m":
        # eq. 2 on the parts truncated under thresholds shared by both parts: one shared block
        assert len(plans) == 1 and plans[0]["kind"] == 5
        assert plans[0]["blocks"] == [(0, n, False)]
    elif mode == "3m_several":
        # one record over the inner order shared by the parts; its blocks tile the inner range
        assert len(plans) == 1 and plans[0]["kind"] == 4
        bl = plans[0]["blocks"]
        assert len(bl) > 1 and bl[0][0] == 0 and bl[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(bl, bl[1:]))
        assert sorted(plans[0]["order"]) == list(range(n))
    else:
        # with the negligible limbs omitted, each real product of this workload is one block
        assert [r["kind"] for r in plans] == [3, 3, 3, 3]
    outs = [to_raw(c) for c in C]
    rng = np.random.default_rng(2048 + structured)
    entries = [(int(a), int(b)) for a, b in zip(rng.integers(0, n, 100), rng.integers(0, n, 100))]
    check_complex(outs, case.A, case.B, n, n, n, p, entries)
    del A, B, C, ws


def test_grouped_batch_sampled(arb):
    cases = grouped_matmuls()
    items = []
    for c in cases:
        items.append(dict(C=arb.Balls.empty(c.N * c.N, (c.prec + 63) // 64),
                          A=arb.Balls.from_raw(c.A[0]), B=arb.Balls.from_raw(c.B[0]), M=c.M,
                          K=c.K, N=c.N, prec=c.prec))
    ctx = arb.default_context()
    arb.mat_mul_batched(items, ctx=ctx)
    assert ctx.status() == 0
    # the block items' plan records, in item order: kind 3 marks an item whose negligible limbs
    # were omitted (its midpoints are then checked against the bound, not bit for bit)
    blocks = [t for t, c in enumerate(cases) if c.M >= 48 and c.K >= 48 and c.N >= 48]
    kinds = dict(zip(blocks, (r["kind"] for r in ctx.last_plans())))
    assert len(kinds) == len(blocks)
    rng = np.random.default_rng(5256)
    checked = {"block": 0, "dot": 0, "p1024": 0}
    picks = list(range(0, len(cases), 4)) + [t for t, c in enumerate(cases) if c.prec == 1024][:12]
    for t in sorted(set(picks)):
        c, it = cases[t], items[t]
        out = to_raw(it["C"])
        nl = (c.prec + 63) // 64
        block = c.M >= 48 and c.K >= 48 and c.N >= 48  # ARBGPU_ALG_AUTO's choice
        ents = [(int(a), int(b)) for a, b in zip(rng.integers(0, c.M, 2), rng.integers(0, c.N, 2))]
        if block and kinds[t] == 3:
            check_bounds(out, c.A[0], c.B[0], c.M, c.K, c.N, c.prec, ents)
            checked["block"] += len(ents)
        elif block:
            check_entries(out, c.A[0], c.B[0], c.M, c.K, c.N, c.prec, ents, nl)
            checked["block"] += len(ents)
        else:
            for i, j in ents:
                ref = alg1.matmul_entry(c.A[0], c.B[0], c.K, c.N, i, j, c.prec, nl)
                assert entry_fields(out, i * c.N + j) == expected_fields(ref, nl), (t, i, j)
                terms = X.matmul_entry_terms(c.A[0], c.B[0], c.K, c.N, i, j)
                S, _Sabs, R = X.dot_terms_exact(terms)
                assert X.contains(X.mid(out, i * c.N + j), X.rad(out, i * c.N + j), S, R)
            checked["dot"] += len(ents)
        if c.prec == 1024:
            checked["p1024"] += len(ents)
    assert sum(checked[k] for k in ("block", "dot")) >= 100
    assert checked["block"] > 0 and checked["dot"] > 0 and checked["p1024"] >= 10
