"""Helpers of the GPU tests: upload seeded inputs, run the library, compare with the oracle."""
from __future__ import annotations

import numpy as np

from synth import RawBalls


def to_raw(balls) -> RawBalls:
    limbs, exp, flags, rman, rexp = balls.to_host()
    return RawBalls(balls.nlimbs, limbs, exp, flags, rman, rexp)


def entry_fields(raw: RawBalls, i: int):
    return ([int(raw.limbs[k, i]) for k in range(raw.nlimbs)], int(raw.exp[i]), int(raw.flags[i]),
            int(raw.rad_man[i]), int(raw.rad_exp[i]))


def expected_fields(res: dict, nlimbs: int):
    limbs = res["limbs"] if res.get("limbs") is not None else [0] * nlimbs
    return (list(limbs), int(res["exp"]), int(res["flags"]), int(res["rad_man"]),
            int(res["rad_exp"]))


def mismatch(raw: RawBalls, i: int, res: dict):
    got = entry_fields(raw, i)
    exp = expected_fields(res, raw.nlimbs)
    return None if got == exp else (got, exp)


def batch_tensors(batch, device="cuda"):
    import torch
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=device)  # noqa
    return dict(xoff=t(batch.xoff, torch.int64), xstep=t(batch.xstep, torch.int64),
                yoff=t(batch.yoff, torch.int64), ystep=t(batch.ystep, torch.int64),
                length=t(batch.length, torch.int64), prec=t(batch.prec, torch.int32),
                sub=t(batch.sub, torch.uint8))


class env:
    """Set environment variables for the duration of a ``with`` block (or a fixture), then
    restore them: the library reads its ARBGPU_* switches on every call."""

    def __init__(self, **values):
        self.values = values
        self.old = {}

    def __enter__(self):
        import os
        for k, v in self.values.items():
            self.old[k] = os.environ.get(k)
            os.environ[k] = v
        return self

    def __exit__(self, *exc):
        import os
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        return False
