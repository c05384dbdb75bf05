"""The seeded generators: normalised layout, correct significant-limb counts, ranges, determinism,
and the recipes of the five workloads (their sizes and value distributions)."""
import inspect

import numpy as np

from oracle import exact as X
from synth import FLAG_ZERO, random_balls
from synth.workloads import (batched_dots, block_matmul_n512, complex_matmul_laplace,
                             dot_matmul_n32_p128, grouped_matmuls, matmul_uniform)


def test_random_balls_layout():
    raw = random_balls(1, 500, 3, np.arange(500) % 192 + 1, -30, 30, rad_bits=100,
                       rad_zero_frac=0.5, zero_frac=0.1)
    for i in range(500):
        fl = int(raw.flags[i])
        if fl & FLAG_ZERO:
            assert X.limb_field(raw, i) == 0
            continue
        v = X.limb_field(raw, i)
        assert v >> 191 == 1  # normalised top limb
        nsig = (fl >> 8) & 0xFF
        low = 3 - nsig
        assert int(raw.limbs[low, i]) != 0 and all(int(raw.limbs[k, i]) == 0 for k in range(low))
        mb = i % 192 + 1
        assert v & ((1 << (192 - mb)) - 1) == 0  # mantissa of at most mb bits
        assert -30 <= int(raw.exp[i]) <= 30
        if raw.rad_man[i]:
            assert int(raw.rad_man[i]) == 1 << 29 and int(raw.rad_exp[i]) == int(raw.exp[i]) - 99


def test_determinism():
    a = matmul_uniform(5, 8, 128, -8, 8)
    b = matmul_uniform(5, 8, 128, -8, 8)
    assert (a.A[0].limbs == b.A[0].limbs).all() and (a.B[0].exp == b.B[0].exp).all()


def test_batched_dots_shapes():
    d = batched_dots(count=100)
    assert d.length.min() >= 1 and d.length.max() <= 256
    assert int(d.length.sum()) == d.x.count == d.y.count
    assert set(np.unique(d.prec)) <= {64, 128, 192}
    # entries of a p=64 dot have one significant limb
    b = int(np.argmax(d.prec == 64))
    o = int(d.xoff[b])
    assert ((d.x.flags[o:o + int(d.length[b])] >> 8) & 0xFF).max() == 1


def test_complex_structured_exponents_follow_inner_index():
    c = complex_matmul_laplace(n=16, structured=True)
    e = c.A[0].exp.reshape(16, 16)
    assert (e.max(axis=0) - e.min(axis=0)).max() <= 8  # same column k: within U[-4,4]


# ---- the workload recipes (shapes, sizes and value distributions the bench and tests rely on)


def _defaults(fn):
    return {k: v.default for k, v in inspect.signature(fn).parameters.items()}


def _nonzero(R):
    return (R.flags & FLAG_ZERO) == 0


def _relative_radius_bits(R):
    """rad_bits with r = 2^(exp - rad_bits) for every nonzero radius (rad_man = 2^29)."""
    nz = R.rad_man != 0
    assert (R.rad_man[nz] == 1 << 29).all()
    return np.unique(R.exp[nz] - R.rad_exp[nz] + 1)


def test_n32dots_recipe():
    c = dot_matmul_n32_p128()
    assert (c.M, c.K, c.N, c.prec) == (32, 32, 32, 128)
    for R in (c.A[0], c.B[0]):
        assert R.nlimbs == 2 and (R.rad_man == 0).all()  # exact balls
        e = R.exp[_nonzero(R)]
        assert e.min() == -8 and e.max() == 8


def test_dots_recipe():
    d = _defaults(batched_dots)
    assert (d["count"], d["len_lo"], d["len_hi"], d["precs"]) == (65536, 1, 256, (64, 128, 192))
    assert (d["exp_lo"], d["exp_hi"], d["rad_zero_frac"]) == (-30, 30, 0.5)
    b = batched_dots(count=3000)
    assert abs(float(b.length.mean()) - 128.5) < 6  # lengths U[1, 256]
    per_p = np.repeat(b.prec.astype(np.int64), b.length)
    for R in (b.x, b.y):
        nz = R.rad_man != 0
        assert 0.45 < float(nz.mean()) < 0.55  # half the radii exactly zero
        assert (R.exp[nz] - R.rad_exp[nz] + 1 == per_p[nz]).all()  # the others 2^-p relative
        assert R.exp.min() >= -30 and R.exp.max() <= 30


def test_n512_recipe():
    assert _defaults(block_matmul_n512)["prec"] == 256
    c = block_matmul_n512()
    assert (c.M, c.K, c.N, c.prec) == (512, 512, 512, 256)
    for R in (c.A[0], c.B[0]):
        assert R.nlimbs == 4
        assert int(R.exp.min()) == -20 and int(R.exp.max()) == 20
        assert (R.rad_man != 0).all() and list(_relative_radius_bits(R)) == [250]
        assert (R.limbs[3] >> np.uint64(63) == 1).all()  # 256-bit mantissas, top bit set


def test_complex2048_recipe():
    d = _defaults(complex_matmul_laplace)
    assert (d["n"], d["prec"], d["scale"], d["clip"], d["rad_bits"]) == (2048, 128, 40.0, 200, 120)
    c = complex_matmul_laplace(n=256)
    e = np.concatenate([R.exp for R in c.A + c.B])
    assert np.abs(e).max() <= 200
    assert 37.0 < float(np.abs(e).mean()) < 43.0  # Laplace(40): E|e| = 40
    for R in c.A + c.B:
        assert list(_relative_radius_bits(R)) == [120]


def test_grouped_recipe():
    d = _defaults(grouped_matmuls)
    assert (d["count"], d["n_lo"], d["n_hi"]) == (256, 16, 512)
    assert d["precs"] == (64, 128, 256, 512, 1024) and (d["exp_lo"], d["exp_hi"]) == (-50, 50)
    cases = grouped_matmuls(count=12, n_hi=40)
    assert len(cases) == 12
    for c in cases:
        assert 16 <= c.N <= 40 and c.M == c.K == c.N and c.prec in d["precs"]
        for R in (c.A[0], c.B[0]):
            assert R.exp.min() >= -50 and R.exp.max() <= 50
            assert list(_relative_radius_bits(R)) == [c.prec - 8]
