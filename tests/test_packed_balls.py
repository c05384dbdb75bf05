"""Host-side layout of ``Balls.packed``: the five arrays are aligned parts of one buffer, a packed
copy moves every field, and the fields read back unchanged (no GPU needed)."""
import numpy as np
import torch

import paper_1901_04289_gb300 as arb
from synth.workloads import matmul_uniform


def test_packed_layout_and_copy():
    case = matmul_uniform(7, 9, 192, -5, 5, rad_bits=180)
    raw = case.A[0]
    a = arb.Balls.from_raw(raw, device="cpu", packed=True)
    ref = arb.Balls.from_raw(raw, device="cpu")
    for x, y in zip(a.tensors(), ref.tensors()):
        assert x.dtype == y.dtype and x.shape == y.shape
        assert torch.equal(x, y)
        assert (x.data_ptr() - a.buffer.data_ptr()) % 256 == 0
    assert a.buffer.numel() >= a.nbytes()
    b = arb.Balls.packed(a.count, a.nlimbs, device="cpu")
    b.copy_from_(a)
    for x, y in zip(b.tensors(), ref.tensors()):
        assert torch.equal(x, y)
    limbs, exp, flags, rman, rexp = b.to_host()
    assert np.array_equal(limbs, np.asarray(raw.limbs, dtype=np.uint64))
    assert np.array_equal(exp, np.asarray(raw.exp))


def test_struct_follows_the_fields():
    """``cstruct`` / ``carray`` keep the C struct between calls and rebuild it as soon as a field's
    data pointer changes, so a call never receives a pointer of a replaced tensor."""
    from paper_1901_04289_gb300 import _carr
    a = arb.Balls.empty(33, 3, device="cpu")
    s1 = a.cstruct()
    assert a.cstruct() is s1 and a.carray() is a.carray()
    fields = ("limbs", "exp", "flags", "rad_man", "rad_exp")
    for name in fields:
        setattr(a, name, getattr(a, name).clone())
        s = a.cstruct()
        assert s is not s1
        assert [getattr(s, f) for f in fields] == [getattr(a, f).data_ptr() for f in fields]
        assert (s.count, s.nlimbs, s.limb_stride) == (33, 3, 33)
        assert _carr([a])[0].exp == a.exp.data_ptr()
        s1 = s
    pair = _carr([a, arb.Balls.empty(33, 3, device="cpu")])
    assert len(pair) == 2 and pair[0].limbs == a.limbs.data_ptr()
