"""The seeded generators: normalised layout, correct significant-limb counts, ranges, determinism."""
import numpy as np

from oracle import exact as X
from synth import FLAG_ZERO, random_balls
from synth.workloads import batched_dots, complex_matmul_laplace, matmul_uniform


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
