"""Seeded synthetic inputs in the ball layout, shared by the tests, the bench and the oracle.

This module only draws random numbers and writes them into the raw ball layout.  It holds none of
the arithmetic of the dot product or of the block matrix multiplication: neither the CUDA path nor
the CPU oracle imports anything from the other, both read what is made here.

Ball layout (one array of `count` entries, the same layout the C library reads):

* ``limbs``  uint64 ``[nlimbs][count]`` -- limb plane ``k`` holds limb ``k`` (little-endian, plane 0 is
  the least significant) of every entry.  A nonzero midpoint is
  ``(-1)^sign * 2^exp * sum_k limbs[k] * 2^(64*(k - nlimbs))`` with bit 63 of the top limb set.
* ``exp``    int64  -- ``2^(exp-1) <= |m| < 2^exp``.
* ``flags``  uint32 -- bit 0 sign, bit 1 zero, bit 2 infinity, bit 3 NaN, bit 4 infinite radius,
  bits 8..15 the number of significant limbs counted from the top down to the lowest nonzero limb.
* ``rad_man`` uint32 and ``rad_exp`` int64 -- radius ``rad_man * 2^(rad_exp - 30)`` with ``rad_man``
  zero or in ``[2^29, 2^30)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FLAG_SIGN = 1
FLAG_ZERO = 2
FLAG_INF = 4
FLAG_NAN = 8
FLAG_RAD_INF = 16
NSIG_SHIFT = 8

SEED_BASE = 1901042890


@dataclass
class RawBalls:
    """Host copy of one ball array in the layout above."""

    nlimbs: int
    limbs: np.ndarray  # uint64 [nlimbs][count]
    exp: np.ndarray  # int64 [count]
    flags: np.ndarray  # uint32 [count]
    rad_man: np.ndarray  # uint32 [count]
    rad_exp: np.ndarray  # int64 [count]

    @property
    def count(self) -> int:
        return int(self.exp.shape[0])

    @staticmethod
    def zeros(count: int, nlimbs: int) -> "RawBalls":
        return RawBalls(
            nlimbs=nlimbs,
            limbs=np.zeros((nlimbs, count), dtype=np.uint64),
            exp=np.zeros(count, dtype=np.int64),
            flags=np.full(count, FLAG_ZERO, dtype=np.uint32),
            rad_man=np.zeros(count, dtype=np.uint32),
            rad_exp=np.zeros(count, dtype=np.int64),
        )

    def take(self, idx) -> "RawBalls":
        idx = np.asarray(idx)
        return RawBalls(self.nlimbs, self.limbs[:, idx].copy(), self.exp[idx].copy(),
                        self.flags[idx].copy(), self.rad_man[idx].copy(), self.rad_exp[idx].copy())

    def nbytes(self) -> int:
        return (self.limbs.nbytes + self.exp.nbytes + self.flags.nbytes + self.rad_man.nbytes
                + self.rad_exp.nbytes)


def _rng(seed) -> np.random.Generator:
    return seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)


def random_balls(seed, count: int, nlimbs: int, mant_bits, exp_lo=None, exp_hi=None, *,
                 exps=None, rad_bits=None, rad_zero_frac: float = 0.0,
                 zero_frac: float = 0.0) -> RawBalls:
    """Random balls: uniform random mantissas of ``mant_bits`` bits (top bit set, the rest uniform),
    random sign, integer exponents uniform in ``[exp_lo, exp_hi]`` (or given by ``exps``).

    ``mant_bits`` is a scalar or a per-entry array (each at most ``64*nlimbs``).  With ``rad_bits``
    set, each radius is ``2^(exp - rad_bits)`` -- an upper bound for ``2^-rad_bits * |m|`` -- and a
    fraction ``rad_zero_frac`` of the radii is exactly zero; without it all radii are zero.  A
    fraction ``zero_frac`` of the midpoints is exactly zero.
    """
    rng = _rng(seed)
    mb = np.broadcast_to(np.asarray(mant_bits, dtype=np.int64), (count,))
    if np.any(mb < 1) or np.any(mb > 64 * nlimbs):
        raise ValueError("mant_bits out of range for nlimbs")
    limbs = rng.integers(0, np.iinfo(np.uint64).max, size=(nlimbs, count), dtype=np.uint64,
                         endpoint=True)
    low_cut = 64 * nlimbs - mb  # bits below this position are zero
    for k in range(nlimbs):
        lo = 64 * k
        cut = np.clip(low_cut - lo, 0, 64)  # number of low bits of limb k to clear
        keep = np.where(cut >= 64, np.uint64(0),
                        ~((np.uint64(1) << cut.astype(np.uint64)) - np.uint64(1)))
        limbs[k] &= keep.astype(np.uint64)
    limbs[nlimbs - 1] |= np.uint64(1) << np.uint64(63)
    if exps is None:
        exp = rng.integers(exp_lo, exp_hi, size=count, endpoint=True).astype(np.int64)
    else:
        exp = np.asarray(exps, dtype=np.int64).copy()
    sign = rng.integers(0, 2, size=count).astype(np.uint32)
    nsig = np.zeros(count, dtype=np.uint32)
    for k in range(nlimbs - 1, -1, -1):
        nsig = np.where(limbs[k] != 0, np.uint32(nlimbs - k), nsig)
    flags = sign | (nsig << np.uint32(NSIG_SHIFT))
    rad_man = np.zeros(count, dtype=np.uint32)
    rad_exp = np.zeros(count, dtype=np.int64)
    if rad_bits is not None:
        nz = rng.random(count) >= rad_zero_frac
        rad_man = np.where(nz, np.uint32(1 << 29), np.uint32(0)).astype(np.uint32)
        rad_exp = np.where(nz, exp - np.int64(rad_bits) + 1, 0).astype(np.int64)
    if zero_frac > 0:
        z = rng.random(count) < zero_frac
        limbs[:, z] = 0
        exp[z] = 0
        flags[z] = FLAG_ZERO
    return RawBalls(nlimbs, limbs, exp, flags.astype(np.uint32), rad_man, rad_exp)


def laplace_exponents(seed, count: int, scale: float, clip: int) -> np.ndarray:
    """Integer exponents drawn from Laplace(0, scale), rounded and clipped to [-clip, clip]."""
    rng = _rng(seed)
    return np.clip(np.rint(rng.laplace(0.0, scale, size=count)), -clip, clip).astype(np.int64)


def concat(parts) -> RawBalls:
    nl = max(p.nlimbs for p in parts)
    out = []
    for p in parts:
        if p.nlimbs < nl:  # widen by zero low limbs: the value is unchanged
            pad = np.zeros((nl - p.nlimbs, p.count), dtype=np.uint64)
            fl = p.flags.copy()
            out.append(RawBalls(nl, np.concatenate([pad, p.limbs], 0), p.exp, fl, p.rad_man,
                                p.rad_exp))
        else:
            out.append(p)
    return RawBalls(nl, np.concatenate([p.limbs for p in out], 1),
                    np.concatenate([p.exp for p in out]), np.concatenate([p.flags for p in out]),
                    np.concatenate([p.rad_man for p in out]),
                    np.concatenate([p.rad_exp for p in out]))
