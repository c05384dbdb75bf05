"""The GPU's reordered, scaled operand copies (csrc/inner_order.cuh, the per-entry body of
`gather_inner_kernel`) run on the host, on the CPU.

For the order and scaling of Section IV-B's inner ordering (``oracle.alg2.inner_order``), every
copied ball must be the original ball times 2^g (A) or 2^-g (B), exactly. The contiguous greedy
plan of the copies (what the GPU planner runs on them) must then be the oracle's ordered plan of
the originals.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from oracle import alg2
from synth import RawBalls
from tests.ballmake import ball_values

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "inner_gather_harness.cu")
BIN = os.path.join(ROOT, "tests", "_build", "inner_gather")
CSRC = os.path.join(ROOT, "paper_1901_04289_gb300", "csrc")


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    srcs = [HARNESS, os.path.join(CSRC, "inner_order.cuh"), os.path.join(CSRC, "common.cuh")]
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(os.path.getmtime(s) for s in srcs):
        os.makedirs(os.path.dirname(BIN), exist_ok=True)
        subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, HARNESS, "-o", BIN],
                       check=True, timeout=600)
    return BIN


def gather(binary, R, rows, K, cols, is_b, order, g):
    ld = cols if is_b else K
    vals = [rows, K, cols, R.nlimbs, int(is_b), ld]
    vals += [int(v) for v in R.limbs.reshape(-1)] + [int(v) for v in R.exp]
    vals += [int(v) for v in R.flags] + [int(v) for v in R.rad_man] + [int(v) for v in R.rad_exp]
    vals += list(order) + list(g)
    out = subprocess.run([binary], input=" ".join(str(v) for v in vals), check=True,
                         capture_output=True, text=True, timeout=120).stdout.splitlines()
    f = {line.split()[0]: [int(v) for v in line.split()[1:]] for line in out}
    n = K * cols if is_b else rows * K
    Y = RawBalls(R.nlimbs, np.array(f["limbs"], dtype=np.uint64).reshape(R.nlimbs, n),
                 np.array(f["exp"], dtype=np.int64), np.array(f["flags"], dtype=np.uint32),
                 np.array(f["rad_man"], dtype=np.uint32), np.array(f["rad_exp"], dtype=np.int64))
    return Y, f["range"][0]


@pytest.mark.parametrize("n", [40, 64])
def test_copies_are_the_scaled_permuted_operands_and_plan_like_the_oracle(harness, n):
    from synth.workloads import complex_matmul_laplace
    case = complex_matmul_laplace(n=n, structured=True)
    A, B = case.A[0], case.B[1]
    M = K = N = n
    order, g = alg2.inner_order(A, B, M, K, N)
    Ao, ra = gather(harness, A, M, K, N, False, order, g)
    Bo, rb = gather(harness, B, M, K, N, True, order, g)
    assert ra == 0 and rb == 0
    for i in range(M):
        for t in range(K):
            k = order[t]
            m, r = ball_values(A, i * K + k)
            mo, ro = ball_values(Ao, i * K + t)
            assert mo == m * Fraction(2) ** g[k] and ro == r * Fraction(2) ** g[k]
    for t in range(K):
        k = order[t]
        for j in range(N):
            m, r = ball_values(B, k * N + j)
            mo, ro = ball_values(Bo, t * N + j)
            assert mo == m * Fraction(2) ** -g[k] and ro == r * Fraction(2) ** -g[k]
    _, blocks = alg2.plan(Ao, Bo, M, K, N, case.prec)
    _, _, _, oblocks = alg2.plan_ordered(A, B, M, K, N, case.prec)
    assert blocks == oblocks


def test_out_of_range_scaling_is_reported(harness):
    from tests.ballmake import make_balls
    A = make_balls([Fraction(3, 4)] * 4)  # 2 x 2, exponent 0
    A.exp[:] = (1 << 60) - 2  # near the fast path's limit
    order, g = [0, 1], [5, 0]  # column 0 moved up by 2^5: out of range
    _, rng = gather(harness, A, 2, 2, 2, False, order, g)
    assert rng == 1
    _, rng = gather(harness, A, 2, 2, 2, False, order, [0, 0])
    assert rng == 0
