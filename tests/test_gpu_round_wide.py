"""The epilogues for long products (more than 16 limbs, p >= 318): the 8-bit warp-MMA
reconstruction (multimodular engine) and the wide CUDA-core one (both engines; ARBGPU_ROUND_MMA=0)
give the same balls, bit for bit, as the general epilogue (ARBGPU_ROUND_WIDE=0 as well), and their
midpoints are the exactly rounded values of the exact products (Algorithm 2 over one block,
Section IV-A), with every ball containing the exact product.

The three cases take the three rounding windows: p = 318 with exponents spread over +-130 (one
block of height about 578, T of about 19 limbs, the 6-limb window), p = 512 (the 10-limb window)
and p = 1024 (the 18-limb window)."""
from __future__ import annotations

import numpy as np
import pytest

from synth import random_balls
from tests.gpu_util import env
from tests.test_gpu_block import check_entries, run_mm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


CASES = [(36, 64, 40, 318, 130, 5), (40, 72, 36, 512, 50, 8), (33, 48, 40, 1024, 50, 16)]


@pytest.mark.parametrize("M,K,N,prec,spread,nl", CASES)
@pytest.mark.parametrize("engine", ["crt", "digits"])
def test_long_epilogues_match_general_and_oracle(arb, M, K, N, prec, spread, nl, engine):
    rng = np.random.default_rng(prec + spread + (engine == "crt"))
    A = random_balls(rng, M * K, nl, 64 * nl - 2, -spread, spread, rad_bits=prec - 8,
                     rad_zero_frac=0.4, zero_frac=0.05)
    B = random_balls(rng, K * N, nl, 64 * nl - 2, -spread, spread, rad_bits=prec - 8,
                     rad_zero_frac=0.4, zero_frac=0.05)
    with env(ARBGPU_ENGINE=engine, ARBGPU_OMIT="0"):
        out, names = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, trace=True)
        plans = arb.default_context().last_plans()
        with env(ARBGPU_ROUND_MMA="0"):
            wide, _ = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK)
            with env(ARBGPU_ROUND_WIDE="0"):
                gen, _ = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK)
    assert "block_round" in names
    assert ("crt_gemm" in names) == (engine == "crt")
    # one exact block
    assert len(plans) == 1 and len(plans[0]["blocks"]) == 1
    for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
        assert np.array_equal(getattr(out, f), getattr(gen, f)), f
        assert np.array_equal(getattr(wide, f), getattr(gen, f)), f
    rng2 = np.random.default_rng(7)
    entries = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 16), rng2.integers(0, N, 16))]
    check_entries(out, A, B, M, K, N, prec, entries, (prec + 63) // 64)


@pytest.mark.parametrize("M,K,N,prec,spread,nl", CASES)
def test_residue_mma_matches_cuda_core_residues(arb, M, K, N, prec, spread, nl):
    """The operands these products take beyond the tensor-core residue kernel get their residues
    from the 8-bit warp-MMA kernel; the CUDA-core residue kernel (ARBGPU_RESIDUE_MMA=0) gives the
    same balls bit for bit, with radii on both sides (the radius operands are written alongside)."""
    rng = np.random.default_rng(3 * prec + spread)
    A = random_balls(rng, M * K, nl, 64 * nl - 2, -spread, spread, rad_bits=prec - 8,
                     rad_zero_frac=0.4, zero_frac=0.05)
    B = random_balls(rng, K * N, nl, 64 * nl - 2, -spread, spread, rad_bits=prec - 8,
                     rad_zero_frac=0.4, zero_frac=0.05)
    with env(ARBGPU_ENGINE="crt", ARBGPU_OMIT="0"):
        out, names = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK, trace=True)
        with env(ARBGPU_RESIDUE_MMA="0"):
            ref, _ = run_mm(arb, A, B, M, K, N, prec, arb.ALG_BLOCK)
    assert "residues_a" in names and "residues_b" in names
    for f in ("limbs", "exp", "flags", "rad_man", "rad_exp"):
        assert np.array_equal(getattr(out, f), getattr(ref, f)), f
    rng2 = np.random.default_rng(11)
    entries = [(int(a), int(b)) for a, b in zip(rng2.integers(0, M, 12), rng2.integers(0, N, 12))]
    check_entries(out, A, B, M, K, N, prec, entries, (prec + 63) // 64)
