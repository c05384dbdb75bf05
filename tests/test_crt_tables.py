"""The multimodular engine's host tables (crt.cu), checked on the CPU against Python integers.

A small harness (``tests/crt_tables_harness.cu``, host code only) prints the tables of one modulus
count.  Every table is checked against what it must satisfy, not against a retyped construction:
* the moduli are the largest primes below 2^16;
* M and its cofactors Q_t = M / m_t are right, and y_t Q_t = 1 (mod m_t);
* the Barrett reciprocals and the GEMM item tables repeat for three products per modulus;
* 2^(32c) mod m_t is right;
* the residue weights' balanced bytes give 2^(8d) (times y_t) mod m_t, and so do the unsigned
  bytes of the warp-MMA residue step;
* the reconstruction weights' balanced bytes sum back to Q_t and M, in BF16 (NM <= 64) and as the
  signed bytes of the warp-MMA reconstruction (every NM), whose offset term is 32896 sum_t Q_t;
* the modulus count covers the requested bits.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "crt_tables_harness.cu")
BIN = os.path.join(ROOT, "tests", "_build", "crt_tables")
CSRC = os.path.join(ROOT, "paper_1901_04289_gb300", "csrc")


@pytest.fixture(scope="module")
def harness():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    srcs = [HARNESS, os.path.join(CSRC, "crt.cu"), os.path.join(CSRC, "internal.h")]
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < max(os.path.getmtime(s) for s in srcs):
        os.makedirs(os.path.dirname(BIN), exist_ok=True)
        subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, HARNESS,
                        os.path.join(CSRC, "crt.cu"), "-o", BIN], check=True, timeout=600)
    return BIN


def tables(binary, NM):
    out = subprocess.run([binary, str(NM)], check=True, capture_output=True, text=True,
                         timeout=60).stdout
    t = {}
    for line in out.splitlines():
        name, *vals = line.split()
        t[name] = [int(v) for v in vals]
    return t


def primes_below_2_16_desc():
    n = 1 << 16
    comp = bytearray(n)
    for i in range(2, int(n ** 0.5) + 1):
        if not comp[i]:
            comp[i * i::i] = b"\x01" * len(comp[i * i::i])
    return [i for i in range(n - 1, 2, -1) if not comp[i]]


def from_limbs(limbs, bits):
    return sum(int(v) << (bits * k) for k, v in enumerate(limbs))


def bf16_value(bits):
    return float(np.array([bits << 16], dtype=np.uint32).view(np.float32)[0])


def balanced_sum(digits):
    return sum(int(d) * 256 ** n for n, d in enumerate(digits))


@pytest.mark.parametrize("NM", [5, 39, 64, 100, 143])
def test_crt_tables(harness, NM):
    t = tables(harness, NM)
    nm, NMW, NCHP, NW32P, NPAD, NQ, NQP = t["dims"]
    assert nm == NM
    mods = t["mods"]
    assert mods == primes_below_2_16_desc()[:NM]
    M = 1
    for m in mods:
        M *= m
    assert NMW == max(2, -(-M.bit_length() // 64))
    assert from_limbs(t["M"], 64) == M and from_limbs(t["M32"], 32) == M
    Q32 = t["Q32"]
    for k, m in enumerate(mods):
        Q = from_limbs(Q32[k * NW32P:(k + 1) * NW32P], 32)
        assert Q == M // m
        assert (t["y"][k] * Q) % m == 1
        assert t["rinv"][k] == int(np.array([1.0 / m], dtype=np.float32).view(np.uint32)[0])
        for c in range(NCHP):
            assert t["pow32"][k * NCHP + c] == pow(2, 32 * c, m)
    # three residue products per modulus in one GEMM batch: item b uses modulus b mod NM
    assert len(t["inv"]) == 3 * NM and len(t["ztab"]) == 4 * 3 * NM
    for b in range(3 * NM):
        m = mods[b % NM]
        assert t["inv"][b] == ((1 << 64) - 1) // m
        f32 = lambda v: int(np.array([v], dtype=np.float32).view(np.uint32)[0])  # noqa: E731
        assert t["ztab"][4 * b:4 * b + 4] == [m, f32(m), f32(1.0 / m), 0]
    # residue weights: row 2t (+1) of side o holds the low (high) balanced byte of the balanced
    # 2^(8d) mod m_t, times y_t for the right-hand side
    w = t["wtab"]
    for side in (0, 1):
        for k, m in enumerate(mods):
            base = (side * NPAD + 2 * k) * 128
            for d in range(128):
                lo, hi = bf16_value(w[base + d]), bf16_value(w[base + 128 + d])
                assert lo == int(lo) and hi == int(hi) and -128 <= lo <= 127
                v = int(256 * hi + lo)
                target = pow(2, 8 * d, m) * (t["y"][k] if side else 1)
                assert (v - target) % m == 0 and abs(v) <= (m - 1) // 2
    # reconstruction weights (NM <= 64): the balanced bytes of each Q_t and of M
    if NM <= 64:
        cw = t["crt_wtab"]
        for k, m in enumerate(mods):
            lo = [bf16_value(cw[n * 128 + 2 * k]) for n in range(NQ)]
            hi = [bf16_value(cw[n * 128 + 2 * k + 1]) for n in range(NQ)]
            assert all(-128 <= v <= 127 and v == int(v) for v in lo)
            assert balanced_sum(lo) == M // m
            assert hi == [0.0] + lo[:-1]  # the high byte of z_t shifts Q_t by one byte
            q1, q256 = bf16_value(cw[NQ * 128 + 2 * k]), bf16_value(cw[NQ * 128 + 2 * k + 1])
            # BF16 keeps 8 significant bits: round to nearest is within 2^-8 relative
            assert abs(q1 - 1 / m) <= 2 ** -8 / m and abs(q256 - 256 / m) <= 2 ** -8 * 256 / m
        mb = [np.array([v], dtype=np.uint32).view(np.float32)[0] for v in t["mbytes"]]
        assert all(-128 <= v <= 127 for v in mb) and balanced_sum([int(v) for v in mb]) == M
        # the q column: with z_t = l + 256 h < m_t, sum_t z_t w_t differs from sum_t z_t / m_t by
        # less than sum_t m_t |w_t - 1/m_t|; with |T / M| < 1/8 its rint is q while that stays
        # below 3/8 (and 256 / m_t's weight is exactly 256 times 1 / m_t's)
        err = Fraction(0)
        for k, m in enumerate(mods):
            w1 = Fraction(bf16_value(cw[NQ * 128 + 2 * k]))
            w256 = Fraction(bf16_value(cw[NQ * 128 + 2 * k + 1]))
            assert w256 == 256 * w1
            err += m * abs(w1 - Fraction(1, m))
        assert err < Fraction(1, 4)
    # the signed-byte table of the warp-MMA reconstruction: column 2t holds the balanced bytes
    # of Q_t, column 2t + 1 the same bytes one place up (the high byte of z_t), zero elsewhere
    K8, NQ8 = t["dims8"]
    w8 = t["w8"]
    assert K8 % 32 == 0 and 2 * NM <= K8 < 2 * NM + 32 and NQ8 % 32 == 0 and NQ <= NQ8
    assert len(w8) == K8 * NQ8 and all(-128 <= v <= 127 for v in w8)
    for k, m in enumerate(mods):
        lo = [w8[n * K8 + 2 * k] for n in range(NQ8)]
        hi = [w8[n * K8 + 2 * k + 1] for n in range(NQ8)]
        assert balanced_sum(lo) == M // m
        assert hi == [0] + lo[:-1]
    assert all(w8[n * K8 + c] == 0 for n in range(NQ8) for c in range(2 * NM, K8))
    # with the z bytes offset by -128, sum_t z_t Q_t = S + 32896 sum_t Q_t
    assert from_limbs(t["c32"], 32) == 32896 * sum(M // m for m in mods)
    assert len(t["c32"]) == 2 * NMW + 2
    # unsigned residue weights of the warp-MMA residue step: column 2t (+1) of side o holds the
    # low (high) byte of 2^(8d) mod m_t (times y_t for o = 1) in row d, zero past 2 NM
    N2, KR = t["dimsr"]
    w8r = t["w8r"]
    assert N2 % 32 == 0 and 2 * NM <= N2 < 2 * NM + 32 and KR % 32 == 0 and KR >= 200
    assert len(w8r) == 2 * N2 * KR and all(0 <= v <= 255 for v in w8r)
    for side in (0, 1):
        for k, m in enumerate(mods):
            base = (side * N2 + 2 * k) * KR
            for d in range(0, KR, 7 if NM > 64 else 1):
                v = w8r[base + d] + 256 * w8r[base + KR + d]
                assert v == pow(2, 8 * d, m) * (t["y"][k] if side else 1) % m
        assert not any(w8r[(side * N2 + c) * KR:(side * N2 + c + 1) * KR] != [0] * KR
                       for c in range(2 * NM, N2))


def test_modulus_count_covers_the_bits(harness):
    t = tables(harness, 5)
    primes = primes_below_2_16_desc()
    for bits, n in zip((100, 600, 2000), t["bits_for"]):
        prod = 1
        for p in primes[:n]:
            prod *= p
        assert prod > 2 ** (bits + 3)  # |T| < M / 8 for every signed `bits`-bit T
        if n > 5:
            prev = prod // primes[n - 1]
            assert prev <= 2 ** (bits + 3)  # and no modulus more than needed


# ---- the residue GEMM's drain: P mod m by Horner's rule in FP32 (crt_gemm_kernel).  Emulated
# here with exact rationals and round-to-nearest-even to 24 bits, on the extreme quarters.

def _f32(x):
    """x (a Fraction) rounded to the nearest float32 value, ties to even (no overflow here)."""
    from fractions import Fraction
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (23 - e)  # 24 significant bits
    v = a * scale
    n, r = divmod(v.numerator, v.denominator)
    twice = 2 * r
    if twice > v.denominator or (twice == v.denominator and n & 1):
        n += 1
    return sign * Fraction(n) / scale


def _drain_mod(D0, D1a, D1b, D2, m):
    from fractions import Fraction
    MAGIC = Fraction(3 * 2**22)
    mf = _f32(Fraction(m))
    rinv = _f32(Fraction(1, m))
    fma = lambda a, b, c: _f32(a * b + c)  # noqa: E731

    def bal(x):
        q = _f32(fma(x, rinv, MAGIC) - MAGIC)
        return fma(-q, mf, x)
    d1 = _f32(bal(Fraction(D1a)) + bal(Fraction(D1b)))
    hi = bal(fma(bal(Fraction(D2)), Fraction(256), d1))
    z = bal(fma(hi, Fraction(256), bal(Fraction(D0))))
    assert z.denominator == 1 and abs(z) <= m // 2 + 2
    r = int(z)
    return r + m if r < 0 else r


def test_float_horner_reduction_of_the_residue_products_is_exact():
    import random
    rnd = random.Random(9)
    top = 1024 * 2**14  # Kp = 1024 products of balanced bytes (one chain of the kernel)
    mods = [65521, 65519, 32771, 40009]
    edge = [top, -top, top - 1, -(top - 1), 0, 1, -1, 2**22, -(2**22)]
    for m in mods:
        cases = [(a, b, c, d) for a in edge[:3] for b in edge[:3] for c in edge[:3]
                 for d in edge[:3]]
        cases += [tuple(rnd.randint(-top, top) for _ in range(4)) for _ in range(300)]
        for D0, D1a, D1b, D2 in cases:
            P = D0 + 256 * (D1a + D1b) + 65536 * D2
            assert _drain_mod(D0, D1a, D1b, D2, m) == P % m, (m, D0, D1a, D1b, D2)
