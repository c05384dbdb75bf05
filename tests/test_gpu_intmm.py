"""The tensor-core integer engine (arbgpu_int_mat_mul) against textbook integer matrix products on
Python integers: bit-exact, including adversarial digits that push every FP32 accumulation chain
to its bound (all digit products equal to 2^14)."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arb():
    import paper_1901_04289_gb300 as arb
    return arb


def to_planes(vals, nl):
    """Python ints (two's complement in 64*nl bits) -> uint64 limb planes [nl][count]."""
    flat = list(vals)
    out = np.zeros((nl, len(flat)), dtype=np.uint64)
    mod = 1 << (64 * nl)
    for i, v in enumerate(flat):
        u = v % mod
        for k in range(nl):
            out[k, i] = (u >> (64 * k)) & 0xFFFFFFFFFFFFFFFF
    return out


def from_planes(planes):
    nl, n = planes.shape
    res = []
    for i in range(n):
        u = 0
        for k in range(nl - 1, -1, -1):
            u = (u << 64) | int(planes[k, i])
        if u >> (64 * nl - 1):
            u -= 1 << (64 * nl)
        res.append(u)
    return res


def run(arb, X, Y, M, K, N, xl, yl, tl):
    import torch
    Xp = torch.from_numpy(to_planes(X, xl).view(np.int64)).cuda()
    Yp = torch.from_numpy(to_planes(Y, yl).view(np.int64)).cuda()
    T = torch.zeros((tl, M * N), dtype=torch.int64, device="cuda")
    arb.int_mat_mul(T, tl, Xp, xl, Yp, yl, M, K, N)
    assert arb.default_context().status() == 0
    return from_planes(T.cpu().numpy().view(np.uint64))


def textbook(X, Y, M, K, N, entries=None):
    if entries is None:
        entries = [(i, j) for i in range(M) for j in range(N)]
    return {(i, j): sum(X[i * K + k] * Y[k * N + j] for k in range(K)) for i, j in entries}


@pytest.mark.parametrize("M,K,N,xl,yl", [(130, 200, 140, 2, 1), (1, 1, 1, 1, 1), (64, 64, 300, 1, 3),
                                         (129, 65, 127, 3, 2)])
def test_random_exact(arb, M, K, N, xl, yl):
    rng = np.random.default_rng(M * 7 + K)
    X = [int(v) for v in rng.integers(-2**62, 2**62, size=M * K)]
    if xl > 1:
        X = [x * (1 << (64 * (xl - 1))) + int(rng.integers(0, 2**62)) for x in X]
    Y = [int(v) for v in rng.integers(-2**62, 2**62, size=K * N)]
    if yl > 1:
        Y = [y * (1 << (64 * (yl - 1))) + int(rng.integers(0, 2**62)) for y in Y]
    tl = xl + yl + 1
    got = run(arb, X, Y, M, K, N, xl, yl, tl)
    ref = textbook(X, Y, M, K, N)
    mod = 1 << (64 * tl)
    for (i, j), v in ref.items():
        assert got[i * N + j] % mod == v % mod, (i, j)


def test_adversarial_digits_fill_every_chain(arb):
    """Balanced digits of -0x80808080808080 are seven -128s; every digit product is 2^14 and every
    256-product accumulation chain reaches exactly 2^22."""
    M, K, N = 128, 512, 128
    v = -0x80808080808080
    X = [v] * (M * K)
    Y = [v] * (K * N)
    got = run(arb, X, Y, M, K, N, 1, 1, 3)
    want = K * v * v
    assert all(g == want for g in got)


def test_sampled_512(arb):
    rng = np.random.default_rng(9)
    M = K = N = 512
    X = [int(a) * (1 << 192) + int(b) for a, b in zip(rng.integers(-2**62, 2**62, M * K),
                                                       rng.integers(0, 2**62, M * K))]
    Y = [int(a) * (1 << 192) + int(b) for a, b in zip(rng.integers(-2**62, 2**62, K * N),
                                                       rng.integers(0, 2**62, K * N))]
    got = run(arb, X, Y, M, K, N, 4, 4, 9)
    pts = [(int(i), int(j)) for i, j in zip(rng.integers(0, M, 300), rng.integers(0, N, 300))]
    ref = textbook(X, Y, M, K, N, pts)
    for (i, j), val in ref.items():
        assert got[i * N + j] == val
