"""arbgpu: ball (midpoint-radius) dot products and matrix multiplication on a GB300 GPU.

Thin Python layer over the C ABI in ``include/arbgpu.h``: ``Balls`` keeps one ball array in device
memory (torch tensors used as plain buffers) and the functions below pass raw pointers, sizes and
the current CUDA stream to ``libarbgpu.so``.  All arithmetic happens in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (ALG_AUTO, ALG_BLOCK, ALG_DOT, MM_COMPLEX_3M, ArbgpuError, CBalls)

__all__ = ["Balls", "Context", "dot", "mat_mul", "int_mat_mul", "ALG_AUTO", "ALG_DOT",
           "ALG_BLOCK", "MM_COMPLEX_3M", "ArbgpuError"]


class Balls:
    """One array of ``count`` balls in device memory, in the layout of ``include/arbgpu.h``.

    ``limbs`` is an int64 tensor ``[nlimbs, count]`` (bit patterns of the uint64 limbs), ``exp`` and
    ``rad_exp`` int64 ``[count]``, ``flags`` and ``rad_man`` int32 ``[count]`` (uint32 bit patterns).
    """

    def __init__(self, limbs, exp, flags, rad_man, rad_exp):
        self.limbs, self.exp, self.flags, self.rad_man, self.rad_exp = limbs, exp, flags, rad_man, \
            rad_exp
        self.nlimbs = int(limbs.shape[0])
        self.count = int(exp.shape[0])

    @staticmethod
    def empty(count, nlimbs, device="cuda"):
        return Balls(torch.zeros((nlimbs, count), dtype=torch.int64, device=device),
                     torch.zeros(count, dtype=torch.int64, device=device),
                     torch.zeros(count, dtype=torch.int32, device=device),
                     torch.zeros(count, dtype=torch.int32, device=device),
                     torch.zeros(count, dtype=torch.int64, device=device))

    @staticmethod
    def packed(count, nlimbs, device="cuda", pin=False):
        """Zero balls whose five arrays are 256-byte aligned parts of one buffer (``buffer``), so
        that the whole array moves between host and device memory in one copy.  ``pin``: pinned
        host memory instead of ``device``."""
        sizes = [8 * nlimbs * count, 8 * count, 4 * count, 4 * count, 8 * count]
        offs, o = [], 0
        for sz in sizes:
            offs.append(o)
            o += (sz + 255) // 256 * 256
        buf = torch.zeros(max(o, 1), dtype=torch.uint8, device="cpu" if pin else device)
        if pin:
            buf = buf.pin_memory()

        def part(i, dt, shape):
            return buf[offs[i]:offs[i] + sizes[i]].view(dt).view(shape)
        b = Balls(part(0, torch.int64, (nlimbs, count)), part(1, torch.int64, (count,)),
                  part(2, torch.int32, (count,)), part(3, torch.int32, (count,)),
                  part(4, torch.int64, (count,)))
        b.buffer = buf
        return b

    @staticmethod
    def from_raw(raw, device="cuda", pin=False, packed=False):
        """Copy a host ball array (numpy fields: limbs, exp, flags, rad_man, rad_exp); with
        ``packed``, into one buffer as ``Balls.packed`` lays it out."""
        if packed:
            limbs = np.ascontiguousarray(raw.limbs)
            b = Balls.packed(int(np.asarray(raw.exp).shape[0]), int(limbs.shape[0]), device, pin)
            for dst, a, dt in ((b.limbs, limbs, np.int64), (b.exp, raw.exp, np.int64),
                               (b.flags, raw.flags, np.int32), (b.rad_man, raw.rad_man, np.int32),
                               (b.rad_exp, raw.rad_exp, np.int64)):
                dst.copy_(torch.from_numpy(np.ascontiguousarray(a).view(dt)))
            return b

        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a).view(dt))
            return x.pin_memory() if pin else x.to(device)
        return Balls(t(raw.limbs, np.int64), t(raw.exp, np.int64), t(raw.flags, np.int32),
                     t(raw.rad_man, np.int32), t(raw.rad_exp, np.int64))

    def to_host(self):
        """(limbs uint64, exp int64, flags uint32, rad_man uint32, rad_exp int64) numpy arrays."""
        return (self.limbs.cpu().numpy().view(np.uint64), self.exp.cpu().numpy(),
                self.flags.cpu().numpy().view(np.uint32), self.rad_man.cpu().numpy().view(np.uint32),
                self.rad_exp.cpu().numpy())

    def copy_from_(self, other, non_blocking=False):
        mine, theirs = getattr(self, "buffer", None), getattr(other, "buffer", None)
        if mine is not None and theirs is not None and mine.numel() == theirs.numel():
            mine.copy_(theirs, non_blocking=non_blocking)  # one copy of the packed buffer
            return self
        for a, b in ((self.limbs, other.limbs), (self.exp, other.exp), (self.flags, other.flags),
                     (self.rad_man, other.rad_man), (self.rad_exp, other.rad_exp)):
            a.copy_(b, non_blocking=non_blocking)
        return self

    def tensors(self):
        return (self.limbs, self.exp, self.flags, self.rad_man, self.rad_exp)

    def nbytes(self):
        return sum(t.numel() * t.element_size() for t in self.tensors())

    def cstruct(self) -> CBalls:
        """The ``arbgpu_balls`` struct of this array.  Kept between calls and rebuilt whenever a
        field's data pointer, the count or the limb count differs from the kept one."""
        key = (self.limbs.data_ptr(), self.exp.data_ptr(), self.flags.data_ptr(),
               self.rad_man.data_ptr(), self.rad_exp.data_ptr(), self.count, self.nlimbs)
        kept = self.__dict__.get("_cstruct")
        if kept is not None and kept[0] == key:
            return kept[1]
        cs = CBalls(key[0], self.count, self.nlimbs, key[1], key[2], key[3], key[4], self.count)
        self._cstruct = (key, cs, (CBalls * 1)(cs))
        return cs

    def carray(self):
        """A one-element ``arbgpu_balls`` array holding ``cstruct()`` (the C calls take arrays)."""
        self.cstruct()
        return self._cstruct[2]


class Context:
    """An ``arbgpu_ctx`` for one device (owns the device status word)."""

    def __init__(self, device=None):
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        h = C.c_void_p()
        rc = _lib.lib().arbgpu_create(C.byref(h), dev)
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_create")
        self.handle = h
        self._ws = None

    def close(self):
        if self.handle is not None:
            _lib.lib().arbgpu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        """Synchronise the stream and return (and clear) the device-side status code."""
        s = _stream_ptr(stream)
        return int(_lib.lib().arbgpu_get_status(self.handle, s))

    def check(self, stream=None):
        rc = self.status(stream)
        if rc != 0:
            raise ArbgpuError(rc, "device status")

    def launch_count(self) -> int:
        n = C.c_int64(0)
        _lib.lib().arbgpu_launch_count(self.handle, C.byref(n))
        return int(n.value)

    def trace(self, enable=True):
        _lib.lib().arbgpu_trace_enable(self.handle, 1 if enable else 0)

    def trace_read(self, max_entries=4096, with_start=False):
        """[(kernel name, device ms, work units)] of the launches traced since the last read
        (with ``with_start``, a fourth field: the start in ms after the first traced launch)."""
        buf = (_lib.CTrace * max_entries)()
        n = C.c_int32(0)
        rc = _lib.lib().arbgpu_trace_read(self.handle, buf, max_entries, C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_trace_read")
        if with_start:
            return [(buf[i].name.decode(), float(buf[i].ms), int(buf[i].units),
                     float(buf[i].start_ms)) for i in range(n.value)]
        return [(buf[i].name.decode(), float(buf[i].ms), int(buf[i].units)) for i in range(n.value)]

    def reserve(self, max_prec, max_inner):
        """Upload every table the block path can need up to these sizes (``arbgpu_reserve``)."""
        rc = _lib.lib().arbgpu_reserve(self.handle, int(max_prec), int(max_inner))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_reserve")

    def set_autotune(self, enable=True):
        """Turn the autotuner on or off (``arbgpu_set_autotune``): the block path's integer engine,
        and the dot / block choice of ALG_AUTO products near the crossover."""
        rc = _lib.lib().arbgpu_set_autotune(self.handle, 1 if enable else 0)
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_set_autotune")

    def autotune_stats(self):
        """dict(buckets, timing_runs, crt_buckets) of the engine autotuner."""
        b, t, c = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        rc = _lib.lib().arbgpu_autotune_stats(self.handle, C.byref(b), C.byref(t), C.byref(c))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_autotune_stats")
        return dict(buckets=b.value, timing_runs=t.value, crt_buckets=c.value)

    def autotune_alg_stats(self):
        """dict(buckets, timing_runs, block_buckets) of the ALG_AUTO dot / block choice."""
        b, t, k = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        rc = _lib.lib().arbgpu_autotune_alg_stats(self.handle, C.byref(b), C.byref(t),
                                                  C.byref(k))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_autotune_alg_stats")
        return dict(buckets=b.value, timing_runs=t.value, block_buckets=k.value)

    def calibrate(self):
        """Measured integer and 8-bit tensor throughput of the device (``arbgpu_calibrate``):
        dict with imad_tops, imad_wide_tops, mma_s8_tops, sm_count, max_clock_mhz."""
        out = _lib.CCalibration()
        rc = _lib.lib().arbgpu_calibrate(self.handle, C.byref(out))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_calibrate")
        return {k: getattr(out, k) for k, _ in _lib.CCalibration._fields_}

    def last_plans(self):
        """The block plans of the last matrix-product call (``arbgpu_last_plans``), one dict per
        real product: kind, h, K, blocks [(start, stop, basecase)], and for kinds 1 and 4 the
        inner order and the scaling exponents."""
        n = C.c_int64(0)
        rc = _lib.lib().arbgpu_last_plans(self.handle, None, 0, C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_last_plans")
        buf = (C.c_int64 * max(1, n.value))()
        rc = _lib.lib().arbgpu_last_plans(self.handle, buf, n.value, C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_last_plans")
        w = list(buf)[:n.value]
        out, q = [], 0
        while q < len(w):
            kind, h, K, nb = w[q:q + 4]
            q += 4
            blocks = [(w[q + 3 * b], w[q + 3 * b + 1], bool(w[q + 3 * b + 2])) for b in range(nb)]
            q += 3 * nb
            rec = dict(kind=kind, h=h, K=K, blocks=blocks)
            if kind in (1, 4):
                rec["order"] = w[q:q + K]
                rec["g"] = w[q + K:q + 2 * K]
                q += 2 * K
            out.append(rec)
        return out

    def workspace(self, nbytes):
        """A cached device buffer of at least ``nbytes`` bytes."""
        if nbytes == 0:
            return None
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws


_default = {}


def default_context(device=None) -> Context:
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _default:
        _default[dev] = Context(dev)
    return _default[dev]


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _pair(b):
    if isinstance(b, (list, tuple)):
        return list(b)
    return [b]


def _arr(structs):
    A = CBalls * len(structs)
    return A(*structs)


def _carr(balls):
    """The ``arbgpu_balls`` array argument for a list of one (real) or two (complex) arrays."""
    if len(balls) == 1:
        return balls[0].carray()
    return _arr([b.cstruct() for b in balls])


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def dot(res, x, y, xoff, xstep, yoff, ystep, length, prec, *, prec_max, len_max, sub=None,
        initial=None, ctx=None, stream=None, approx=False, reduce_prec=False):
    """Batched ball dots (``arbgpu_dot_ex``): with ``approx`` the same midpoints and zero radii
    (``arbgpu_approx_dot``); with ``reduce_prec`` the precision reduction ("optimize p") of Section III-C.
    ``res``, ``x``, ``y``, ``initial``: a ``Balls`` (real) or a pair ``(re, im)`` (complex).  Index
    arrays: int64 device tensors; ``prec`` int32; ``sub`` uint8 or None."""
    ctx = ctx or default_context()
    cplx = isinstance(x, (list, tuple))
    r, xs, ys = _pair(res), _pair(x), _pair(y)
    init = _pair(initial) if initial is not None else None
    batch = int(length.shape[0])
    options = (1 if approx else 0) | (2 if reduce_prec else 0)
    rc = _lib.lib().arbgpu_dot_ex(
        ctx.handle, _carr(r), _carr(init) if init else None, _ptr(sub),
        _carr(xs), _ptr(xoff), _ptr(xstep), _carr(ys),
        _ptr(yoff), _ptr(ystep), _ptr(length), _ptr(prec), batch, int(prec_max), int(len_max),
        1 if cplx else 0, options, None, 0, _stream_ptr(stream))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_dot_ex")


def mat_mul_workspace_size(M, K, N, prec, a_nlimbs, b_nlimbs, complex_mode=False, alg=ALG_AUTO,
                           flags=0, ctx=None):
    ctx = ctx or default_context()
    n = C.c_size_t(0)
    rc = _lib.lib().arbgpu_mat_mul_workspace_size(ctx.handle, M, K, N, prec, a_nlimbs, b_nlimbs,
                                                  1 if complex_mode else 0, alg, flags,
                                                  C.byref(n))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_mat_mul_workspace_size")
    return int(n.value)


def mat_mul(C_out, A, B, M, K, N, prec, *, alg=ALG_AUTO, flags=0, lda=None, ldb=None, ldc=None,
            workspace=None, ctx=None, stream=None):
    """Ball matrix product ``C = A * B`` (``arbgpu_mat_mul``); complex when A is a pair.

    ``A`` is M x K, ``B`` K x N, ``C_out`` M x N, row-major with leading dimensions ``lda``, ``ldb``,
    ``ldc`` (default K, N, N).  ``alg``: ``ALG_AUTO`` (Algorithm 2 from M, K, N >= 48, dots below),
    ``ALG_DOT`` (one Algorithm 1 dot per entry) or ``ALG_BLOCK`` (Algorithm 2).  ``flags``: 0 or
    ``MM_COMPLEX_3M`` (complex midpoints by eq. 2 when the parts share one scaling in a single
    block).  ``workspace``: a device tensor of at least ``mat_mul_workspace_size`` bytes for the
    same arguments, else one cached in the context is used."""
    ctx = ctx or default_context()
    cplx = isinstance(A, (list, tuple))
    cs, As, Bs = _pair(C_out), _pair(A), _pair(B)
    lda = K if lda is None else lda
    ldb = N if ldb is None else ldb
    ldc = N if ldc is None else ldc
    if workspace is None and alg != ALG_DOT:  # (the classical algorithm needs none)
        need = mat_mul_workspace_size(M, K, N, prec, max(a.nlimbs for a in As),
                                      max(b.nlimbs for b in Bs), cplx, alg, flags, ctx)
        workspace = ctx.workspace(need)
    wsp = _ptr(workspace)
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = _lib.lib().arbgpu_mat_mul(ctx.handle, _carr(cs), _carr(As), _carr(Bs), M, K, N, lda, ldb,
                                   ldc, prec, 1 if cplx else 0, alg, flags, wsp, wsb,
                                   _stream_ptr(stream))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_mat_mul")


def mat_mul_batched(items, *, workspace=None, ctx=None, stream=None):
    """Grouped batch of ball matrix products (``arbgpu_mat_mul_batched``).  ``items``: list of
    dicts with keys C, A, B (Balls or (re, im) pairs), M, K, N, prec and optional alg, flags
    (``MM_COMPLEX_3M``), lda, ldb, ldc.  Small classical items run in one grouped launch, the
    others by the block algorithm."""
    ctx = ctx or default_context()
    arr = (_lib.CMatmulDesc * len(items))()
    for q, it in enumerate(items):
        cs, As, Bs = _pair(it["C"]), _pair(it["A"]), _pair(it["B"])
        cplx = len(As) == 2
        d = arr[q]
        for r in range(2):
            src = r if cplx else 0
            d.C[r] = cs[src].cstruct()
            d.A[r] = As[src].cstruct()
            d.B[r] = Bs[src].cstruct()
        d.M, d.K, d.N = it["M"], it["K"], it["N"]
        d.lda = it.get("lda", it["K"])
        d.ldb = it.get("ldb", it["N"])
        d.ldc = it.get("ldc", it["N"])
        d.prec = it["prec"]
        d.complex_mode = 1 if cplx else 0
        d.alg = it.get("alg", ALG_AUTO)
        d.flags = it.get("flags", 0)
    if workspace is None:
        n = C.c_size_t(0)
        rc = _lib.lib().arbgpu_mat_mul_batched_workspace_size(ctx.handle, arr, len(items),
                                                              C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_mat_mul_batched_workspace_size")
        workspace = ctx.workspace(int(n.value))
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = _lib.lib().arbgpu_mat_mul_batched(ctx.handle, arr, len(items), _ptr(workspace), wsb,
                                           _stream_ptr(stream))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_mat_mul_batched")


def int_mat_mul(T, t_limbs, X, x_limbs, Y, y_limbs, M, K, N, *, workspace=None, ctx=None,
                stream=None):
    """Exact integer matrix product over limb planes (``arbgpu_int_mat_mul``)."""
    ctx = ctx or default_context()
    if workspace is None:
        n = C.c_size_t(0)
        rc = _lib.lib().arbgpu_int_mat_mul_workspace_size(ctx.handle, x_limbs, y_limbs, M, K, N,
                                                          C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_int_mat_mul_workspace_size")
        workspace = ctx.workspace(int(n.value))
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = _lib.lib().arbgpu_int_mat_mul(ctx.handle, _ptr(T), t_limbs, _ptr(X), x_limbs, _ptr(Y),
                                       y_limbs, M, K, N, _ptr(workspace), wsb, _stream_ptr(stream))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_int_mat_mul")


def series_exp(res, a, length, batch, prec, *, workspace=None, ctx=None, stream=None):
    """Power series exponential of ``batch`` series (``arbgpu_series_exp``): coefficient k of
    series s at index k * batch + s of ``a`` and ``res``."""
    ctx = ctx or default_context()
    if workspace is None:
        n = C.c_size_t(0)
        rc = _lib.lib().arbgpu_series_exp_workspace_size(ctx.handle, length, batch, prec,
                                                         C.byref(n))
        if rc != 0:
            raise ArbgpuError(rc, "arbgpu_series_exp_workspace_size")
        workspace = ctx.workspace(int(n.value))
    wsb = 0 if workspace is None else workspace.numel() * workspace.element_size()
    r, x = res.cstruct(), a.cstruct()
    rc = _lib.lib().arbgpu_series_exp(ctx.handle, C.byref(r), C.byref(x), length, batch, prec,
                                      _ptr(workspace), wsb, _stream_ptr(stream))
    if rc != 0:
        raise ArbgpuError(rc, "arbgpu_series_exp")
