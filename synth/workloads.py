"""The synthetic workloads, each built from a fixed seed.

Every workload mirrors the "uniform p-bit entries" inputs the paper benchmarks (Section V), with the
sizes, precisions, exponent distributions and radii listed below.  Matrices are row-major: entry
(i, k) of an M x K matrix is index ``i*K + k`` of its ball array.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import SEED_BASE, RawBalls, concat, laplace_exponents, random_balls


@dataclass
class MatmulCase:
    name: str
    M: int
    K: int
    N: int
    prec: int
    A: list  # [re] or [re, im] RawBalls, M*K entries
    B: list  # [re] or [re, im] RawBalls, K*N entries
    meta: dict = field(default_factory=dict)

    @property
    def complex(self) -> bool:
        return len(self.A) == 2


@dataclass
class DotBatch:
    name: str
    x: RawBalls
    y: RawBalls
    xoff: np.ndarray
    xstep: np.ndarray
    yoff: np.ndarray
    ystep: np.ndarray
    length: np.ndarray
    prec: np.ndarray
    sub: np.ndarray
    initial: RawBalls | None = None


def limbs_for(bits: int) -> int:
    return (bits + 63) // 64


def matmul_uniform(seed, n, prec, exp_lo, exp_hi, rad_bits=None, mant_bits=None, m=None, k=None,
                   name="") -> MatmulCase:
    """Real ball matrices with uniform random ``mant_bits``-bit mantissas (default ``prec``),
    exponents uniform in ``[exp_lo, exp_hi]`` and radii ``2^-rad_bits`` relative (or zero)."""
    rng = np.random.default_rng(seed)
    m = n if m is None else m
    k = n if k is None else k
    mb = prec if mant_bits is None else mant_bits
    nl = limbs_for(mb)
    A = random_balls(rng, m * k, nl, mb, exp_lo, exp_hi, rad_bits=rad_bits)
    B = random_balls(rng, k * n, nl, mb, exp_lo, exp_hi, rad_bits=rad_bits)
    return MatmulCase(name or f"real matmul {m}x{k}x{n} p={prec}", m, k, n, prec, [A], [B])


def dot_matmul_n32_p128(seed=SEED_BASE + 1) -> MatmulCase:
    """Real N=32, p=128: 128-bit mantissas, exponents in [-8, 8], exact (zero-radius) balls."""
    return matmul_uniform(seed, 32, 128, -8, 8, None, name="real ball matmul N=32 p=128 (dots)")


def batched_dots(seed=SEED_BASE + 2, count=65536, len_lo=1, len_hi=256, precs=(64, 128, 192),
                 exp_lo=-30, exp_hi=30, rad_zero_frac=0.5) -> DotBatch:
    """Batched real dots of uniform random length in [len_lo, len_hi]; each dot has its own precision
    p drawn from ``precs`` and p-bit mantissas, exponents uniform in [exp_lo, exp_hi], radii
    ``2^-p`` relative with a fraction ``rad_zero_frac`` exactly zero.  x and y are separate arrays
    and every term is read once (unit strides)."""
    rng = np.random.default_rng(seed)
    length = rng.integers(len_lo, len_hi, size=count, endpoint=True).astype(np.int64)
    prec = rng.choice(np.asarray(precs, dtype=np.int32), size=count).astype(np.int32)
    off = np.zeros(count, dtype=np.int64)
    off[1:] = np.cumsum(length)[:-1]
    total = int(length.sum())
    per_entry_p = np.repeat(prec.astype(np.int64), length)
    nl = limbs_for(max(precs))
    x = random_balls(rng, total, nl, per_entry_p, exp_lo, exp_hi, rad_bits=None)
    y = random_balls(rng, total, nl, per_entry_p, exp_lo, exp_hi, rad_bits=None)
    # radius 2^(e - p) per entry, half of them zero
    for r in (x, y):
        nz = rng.random(total) >= rad_zero_frac
        r.rad_man = np.where(nz, np.uint32(1 << 29), np.uint32(0)).astype(np.uint32)
        r.rad_exp = np.where(nz, r.exp - per_entry_p + 1, 0).astype(np.int64)
    ones = np.ones(count, dtype=np.int64)
    return DotBatch(f"batched real ball dots: {count} dots, length U[{len_lo},{len_hi}], "
                    f"p in {tuple(precs)}", x, y, off.copy(), ones.copy(), off.copy(), ones.copy(),
                    length, prec, np.zeros(count, dtype=np.uint8))


def block_matmul_n512(seed=SEED_BASE + 3, prec=256) -> MatmulCase:
    """Real N=512: ``prec``-bit mantissas, exponents in [-20, 20], radii 2^-250 relative (the same
    draw is used at p=128 with 128-bit mantissas for the block-versus-dot comparison)."""
    return matmul_uniform(seed, 512, prec, -20, 20, rad_bits=250,
                          name=f"real ball matmul N=512 p={prec}")


def complex_matmul_laplace(seed=SEED_BASE + 4, n=2048, prec=128, scale=40.0, clip=200,
                           rad_bits=120, structured=False) -> MatmulCase:
    """Complex N x N, p=128 mantissas for both parts, radii 2^-120 relative.

    Literal variant: every entry's exponent is drawn i.i.d. from Laplace(0, scale), rounded and
    clipped to [-clip, clip].  Structured variant: the exponent of A[i,k] is c_k + U[-4,4] and of
    B[k,j] is c'_k + U[-4,4] with c_k, c'_k ~ Laplace(0, scale) clipped, so that the inner index
    carries the magnitude variation and contiguous exponent blocks form."""
    rng = np.random.default_rng(seed)
    nl = limbs_for(prec)
    mats = []
    for which in ("A", "B"):
        parts = []
        for _part in ("re", "im"):
            if structured:
                c = laplace_exponents(rng, n, scale, clip)
                jitter = rng.integers(-4, 4, size=(n, n), endpoint=True)
                if which == "A":
                    e = np.clip(c[None, :] + jitter, -clip, clip)  # A[i,k]: varies with k
                else:
                    e = np.clip(c[:, None] + jitter, -clip, clip)  # B[k,j]: varies with k
                e = e.reshape(-1)
            else:
                e = laplace_exponents(rng, n * n, scale, clip)
            parts.append(random_balls(rng, n * n, nl, prec, exps=e, rad_bits=rad_bits))
        mats.append(parts)
    kind = "structured" if structured else "literal"
    return MatmulCase(f"complex ball matmul N={n} p={prec} Laplace({scale:g}) exponents ({kind})",
                      n, n, n, prec, mats[0], mats[1], meta={"structured": structured})


def grouped_matmuls(seed=SEED_BASE + 5, count=256, n_lo=16, n_hi=512,
                    precs=(64, 128, 256, 512, 1024), exp_lo=-50, exp_hi=50) -> list:
    """``count`` independent real square matmuls, N uniform in [n_lo, n_hi], p drawn from ``precs``,
    p-bit mantissas, exponents uniform in [exp_lo, exp_hi], radii 2^-(p-8) relative."""
    rng = np.random.default_rng(seed)
    cases = []
    for t in range(count):
        n = int(rng.integers(n_lo, n_hi, endpoint=True))
        p = int(rng.choice(precs))
        sub = int(rng.integers(0, 2**62))
        cases.append(matmul_uniform(sub, n, p, exp_lo, exp_hi, rad_bits=p - 8,
                                    name=f"group item {t}: N={n} p={p}"))
    return cases


__all__ = ["MatmulCase", "DotBatch", "matmul_uniform", "dot_matmul_n32_p128", "batched_dots",
           "block_matmul_n512", "complex_matmul_laplace", "grouped_matmuls", "limbs_for", "concat"]
