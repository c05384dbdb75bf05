"""The host side of the GPU's inner ordering (csrc/inner_order.cu) against the oracle's restatement
of the same reading (``oracle.alg2.inner_order``), on the CPU.

The per-index tops a_k, b_k that the GPU takes from its entry scan are formed here from the
oracle's decoded entries (the largest exponent of column k of A and of row k of B). The harness
turns them into the order and the inner scaling, which must equal the oracle's.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import zlib

import numpy as np
import pytest

from oracle import alg2
from synth import random_balls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "inner_order_harness.cu")
BIN = os.path.join(ROOT, "tests", "_build", "inner_order")
CSRC = os.path.join(ROOT, "paper_1901_04289_gb300", "csrc")
INT64_MIN = -(1 << 63)


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    srcs = [HARNESS, os.path.join(CSRC, "inner_order.cu"), os.path.join(CSRC, "internal.h")]
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(os.path.getmtime(s) for s in srcs):
        os.makedirs(os.path.dirname(BIN), exist_ok=True)
        subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, HARNESS,
                        os.path.join(CSRC, "inner_order.cu"), "-o", BIN], check=True, timeout=600)
    return BIN


def gpu_rule(binary, a, b):
    inp = " ".join(str(v) for v in [len(a)] + list(a) + list(b))
    out = subprocess.run([binary], input=inp, check=True, capture_output=True, text=True,
                         timeout=60).stdout.splitlines()
    ord_ = [int(v) for v in out[0].split()[1:]]
    g = [int(v) for v in out[1].split()[1:]]
    return ord_, g


def tops(A, B, M, K, N):
    a, b = [], []
    for k in range(K):
        ta = [alg2.top_bottom(A, i * K + k) for i in range(M)]
        tb = [alg2.top_bottom(B, k * N + j) for j in range(N)]
        ta = [t[0] for t in ta if t is not None]
        tb = [t[0] for t in tb if t is not None]
        a.append(max(ta) if ta else INT64_MIN)
        b.append(max(tb) if tb else INT64_MIN)
    return a, b


def _case(kind):
    from synth.workloads import complex_matmul_laplace
    rng = np.random.default_rng(zlib.crc32(kind.encode()))
    if kind == "structured":
        case = complex_matmul_laplace(n=64, structured=True)
        return case.A[0], case.B[1], 64, 64, 64
    if kind == "ties":  # equal a_k + b_k everywhere: the order falls back to the index
        M, K, N = 3, 40, 2
        return (random_balls(rng, M * K, 1, 64, 0, 0), random_balls(rng, K * N, 1, 64, 0, 0),
                M, K, N)
    M, K, N = 4, 50, 3  # zeros: dead indices, odd differences b_k - a_k of both signs
    A = random_balls(rng, M * K, 1, 64, -300, 300, zero_frac=0.5)
    B = random_balls(rng, K * N, 1, 64, -300, 300, zero_frac=0.5)
    return A, B, M, K, N


@pytest.mark.parametrize("kind", ["structured", "ties", "zeros"])
def test_host_order_equals_the_oracle(harness, kind):
    A, B, M, K, N = _case(kind)
    a, b = tops(A, B, M, K, N)
    ord_, g = gpu_rule(harness, a, b)
    oo, og = alg2.inner_order(A, B, M, K, N)
    assert ord_ == oo and g == og
    if kind == "zeros":
        assert any(v == INT64_MIN for v in a + b)  # the case really has dead indices
        assert any(g[k] < 0 and (b[k] - a[k]) % 2 for k in range(K))  # floor of a negative odd
