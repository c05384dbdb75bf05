"""Benchmark: effective ball multiply-add rate of the real ball matrix product at N=512.

Workload (default): real ball matrices A, B of size 512 x 512, uniform random 256-bit mantissas,
exponents uniform in [-20, 20], radii 2^-250 relative, multiplied at p = 256 with the library's
default algorithm (the block algorithm of Section IV-A once available, else the classical
dot-product algorithm).  The same inputs with 128-bit mantissas are timed at p = 128, and both
precisions are also timed with the classical warp-per-dot algorithm, so the line reports the
block-versus-dot speedup at p = 128 and p = 256.

One step = one complete ``arbgpu_mat_mul`` call (every kernel of the path) on inputs resident in
device memory; L2 is flushed (512 MiB write) before each timed step and the step is timed with CUDA
events on the launching stream.  ``e2e`` repeats the measurement through the same public call with
the inputs copied from pinned host memory and the result copied back inside the timed region.

``--impl reference`` times the CPU oracle (exact rational dot products on Python integers, then one
rounding) on a bounded sample of output entries of the same workload.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]
       (N > 1 under torchrun: every rank runs its own replica; weak scaling)
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
METRIC = "ball matmul eff. GMAC/s at p=128/256 vs plain dot path; INT8 TC % of peak"
UNIT = "GMAC/s"
N_DEFAULT = 512


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def workload_name(n, prec):
    return (f"real ball matmul N={n} p={prec}: uniform {prec}-bit mantissas, exponents U[-20,20], "
            f"radii 2^-250 relative")


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while active."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                maxs.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sms:
            return None
        top = max(sms)
        load = [s for s in sms if s >= 0.5 * top] or sms
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


# --------------------------------------------------------------------------- rooflines

IMAD_PER_CLK_PER_SM = 64  # 32-bit integer multiply(-add) issue rate per SM per clock
SMS = 152
# the device's measured 32-bit multiply-add rate (arbgpu_calibrate), set once per run
MEASURED_ALU = {}


def measure_alu(ctx):
    """Run the library's calibration kernels once; their IMAD rate becomes the ALU peak."""
    try:
        MEASURED_ALU.update(ctx.calibrate())
    except Exception as e:  # the derived figure stands in, and the line says so
        MEASURED_ALU["error"] = str(e)
    return dict(MEASURED_ALU)


def alu_peak_of(sm_mhz):
    """(peak in T 32-bit multiply-adds/s, where it comes from): the rate arbgpu_calibrate measured
    on this device, else unit counts x the sampled SM clock."""
    if MEASURED_ALU.get("imad_tops"):
        return MEASURED_ALU["imad_tops"], "measured: arbgpu_calibrate mad.lo.u32 rate"
    return (SMS * IMAD_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12,
            f"derived: {SMS} SMs x {IMAD_PER_CLK_PER_SM} IMAD/clk x {sm_mhz:.0f} MHz")


def kernel_summary(recs, step_ms_total):
    per = {}
    for name, kms, units in recs:
        d = per.setdefault(name, [0.0, 0, 0])
        d[0] += kms
        d[1] += 1
        d[2] += units
    return {k: {"launches": v[1], "ms_total": round(v[0], 4),
                "share": round(v[0] / step_ms_total, 4) if step_ms_total else None,
                "units": v[2]} for k, v in per.items()}


def roofline_of(name, k, peaks, sm_mhz, limb_n=None):
    """Roofline entry of one kernel from its trace totals (ms_total, launches, units).  For the
    fused dot kernel (units = terms) `limb_n` gives the limbs per factor: 4 n^2 32-bit multiplies
    per term."""
    avg_s = k["ms_total"] / k["launches"] * 1e-3
    units = k["units"] / k["launches"]
    alu_peak, alu_source = alu_peak_of(sm_mhz)
    if name in ("dot_fused", "dot_tile") and limb_n:
        achieved = 4 * limb_n * limb_n * units / avg_s / 1e12
        return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": alu_peak,
                "unit": "T int32-mul/s", "frac": achieved / alu_peak, "traffic": None,
                "work": f"{units:.4g} terms per launch x {4 * limb_n * limb_n} 32-bit multiplies",
                "peak_source": alu_source}
    if name in ("crt_gemm", "digit_gemm", "digit_gemm_mid", "digit_gemm_rad"):
        achieved = 2.0 * units / avg_s / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)
        return {"bound": "tensor", "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "note": "exact BF16 digit products (1 digit MAC = 2 flops) vs the measured "
                        "dense BF16 burst peak (no INT8 tcgen05 on sm_103a)"}
    if name == "residues":  # units: algorithmic bytes (operands read, residue planes written)
        achieved = units / avg_s / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                "work": f"{units:.4g} bytes per launch: every operand entry read once, every "
                        "residue and radius-operand plane written once"}
    if name in ("block_round", "residues_a", "residues_b"):
        achieved = units / avg_s / 1e12
        return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": alu_peak,
                "unit": "T int32-mul/s", "frac": achieved / alu_peak, "traffic": None,
                "peak_source": alu_source,
                "work": "CRT sums (block_round) / residue chunks (residues): 32-bit "
                        "multiply-adds per launch"}
    return {"kernel": name, "ms_avg": avg_s * 1e3}


DOT_KERNELS = ("dot_setup", "dot_eval", "dot_fused", "dot_tile")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the headline workload's
# kernels (N = 512, p = 256: residue_tc_kernel, crt_gemm_kernel and crt_round_tc_kernel, the last
# traced as block_round), from the ncu capture summarised in
# profiles/multimodular_n512_p256_full.md; valid only for that workload and for kernels unchanged
# since that capture.
TRAFFIC_N512_P256 = {"crt_gemm": 88.24e6, "residues": 58.76e6, "block_round": 24.28e6}

# steps of the end-to-end arm's timed region (at least): the pipeline's fill and drain, about one
# step's upload plus one product and read-back, are spread over that many steps
E2E_MIN_STEPS = 100


def dot_work(terms_by_n, unique_bytes=None):
    """Algorithmic work of a dot-path call: terms_by_n maps limbs read per factor (n) to the number
    of terms.  mults = 4 n^2 32-bit multiplies per term (n^2 64x64->128-bit limb products);
    bytes = every input byte the terms need, once: 2 (8n + 24) per term for independent dots, or
    `unique_bytes` when entries are shared between dots (a matrix product)."""
    terms = sum(terms_by_n.values())
    mults = sum(4 * n * n * t for n, t in terms_by_n.items())
    byts = unique_bytes if unique_bytes is not None else sum(
        2 * (8 * n + 24) * t for n, t in terms_by_n.items())
    return {"terms": terms, "mults": mults, "bytes": byts}


def dot_roofline(kernels, work, calls, peaks, sm_mhz):
    """Roofline of the dot path over the timed region: one fused launch, or one setup launch and
    one launch per size class, each call.  The bound is whichever of HBM bytes or integer multiplies takes longer at
    peak; `achieved` divides the work of one call by the device time of one call."""
    t_eval = (kernels.get("dot_eval", {}).get("ms_total", 0.0) +
              kernels.get("dot_fused", {}).get("ms_total", 0.0) +
              kernels.get("dot_tile", {}).get("ms_total", 0.0)) * 1e-3 / calls
    t_set = kernels.get("dot_setup", {}).get("ms_total", 0.0) * 1e-3 / calls
    t_all = t_eval + t_set
    if t_all <= 0:
        return None
    alu_peak, alu_source = alu_peak_of(sm_mhz)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    t_hbm = work["bytes"] / (hbm_peak * 1e9)
    t_alu = work["mults"] / (alu_peak * 1e12)
    names = [k for k in ("dot_setup", "dot_eval", "dot_fused", "dot_tile") if k in kernels]
    base = {"kernel": " + ".join(names), "ms_per_call": t_all * 1e3,
            "eval_ms_per_call": t_eval * 1e3, "terms_per_call": work["terms"],
            "traffic": None}
    if t_hbm >= t_alu:
        achieved = work["bytes"] / t_all / 1e9
        base.update({"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "bytes_per_call": work["bytes"],
                     "peak_source": "measured copy bandwidth"})
    else:
        achieved = work["mults"] / t_eval / 1e12
        base.update({"bound": "alu", "achieved": achieved, "peak": alu_peak,
                     "unit": "T int32-mul/s", "frac": achieved / alu_peak,
                     "mults_per_call": work["mults"],
                     "peak_source": alu_source})
    return base


# --------------------------------------------------------------------------- replicas

def replica_throughput(ms, units, world, device="cpu"):
    """Whole-job rate of `world` independent replicas that each processed `units` work units in
    `ms` milliseconds: the slowest rank's time (max over ranks through torch.distributed when
    world > 1) sets the job time.  Returns (ms_max, units per second / 1e9 over all ranks)."""
    import torch
    import torch.distributed as dist
    tot = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    ms_max = float(tot.item())
    return ms_max, world * units / (ms_max * 1e-3) / 1e9


# --------------------------------------------------------------------------- oracle arm

def oracle_sample(case, prec, entries, seconds):
    """Time the oracle's exact definition on sampled output entries; returns (MAC/s, entries)."""
    from oracle import exact as X
    import numpy as np
    rng = np.random.default_rng(0)
    K, N = case.K, case.N
    done = 0
    macs = 0
    t0 = time.perf_counter()
    while done < entries and (time.perf_counter() - t0) < seconds:
        i, j = int(rng.integers(case.M)), int(rng.integers(N))
        terms = X.matmul_entry_terms(case.A[0], case.B[0], K, N, i, j)
        X.result_exact(terms, prec, (prec + 63) // 64)
        done += 1
        macs += K
    dt = time.perf_counter() - t0
    return macs / dt, done, dt


def _oracle_worker(job):
    """One host process of the oracle timing: rebuild the seeded workload, then time the oracle's
    exact definition on random output entries for `seconds`; returns (MACs, seconds, entries)."""
    prec, n, seconds, seed = job
    from synth.workloads import block_matmul_n512, matmul_uniform
    case = (block_matmul_n512(prec=prec) if n == N_DEFAULT
            else matmul_uniform(1901042893, n, prec, -20, 20, rad_bits=250))
    from oracle import exact as X
    import numpy as np
    rng = np.random.default_rng(seed)
    done = macs = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        i, j = int(rng.integers(case.M)), int(rng.integers(case.N))
        X.result_exact(X.matmul_entry_terms(case.A[0], case.B[0], case.K, case.N, i, j), prec,
                       (prec + 63) // 64)
        done += 1
        macs += case.K
    return macs, time.perf_counter() - t0, done


def oracle_all_cores(prec, n, seconds, pool, cores):
    """The oracle on every host core at once (one spawned process per core, each on its own
    random entries); returns (MAC/s summed over the processes, entries, seconds)."""
    res = pool.map(_oracle_worker, [(prec, n, seconds, 1000 + c) for c in range(cores)])
    rate = sum(m / dt for m, dt, _ in res)
    return rate, sum(e for _, _, e in res), max(dt for _, dt, _ in res)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import multiprocessing as mp
    from synth.workloads import block_matmul_n512
    case = block_matmul_n512(prec=args.prec)
    cores = host_cores()
    # each step: every host core runs the oracle on its own random entries for a bounded time
    step_s = max(1.0, min(10.0, 60.0 / max(args.steps + args.warmup, 1)))
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_all_cores(args.prec, case.N, 0.5, pool, cores)
        rates = []
        ents = 0
        secs = 0.0
        for _ in range(args.steps):
            r, n, dt = oracle_all_cores(args.prec, case.N, step_s, pool, cores)
            rates.append(r)
            ents += n
            secs += dt
    value = statistics.mean(rates) / 1e9
    sample = (f"{ents} output entries of the {case.N}x{case.N} product ({case.K} terms each) on "
              f"{cores} processes, {args.steps} steps of {step_s:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "exact (python int)",
            "data": "synthetic", "config": {"workload": workload_name(case.N, args.prec),
                                            "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- other workloads

def run_workload(args):
    """One JSON line for one of the non-headline workloads (single GPU)."""
    import numpy as np
    import torch

    import paper_1901_04289_gb300 as arb
    from oracle import exact as X
    from synth import SEED_BASE
    from synth.workloads import (batched_dots, complex_matmul_laplace, dot_matmul_n32_p128,
                                 grouped_matmuls, matmul_uniform)
    from tests.gpu_util import batch_tensors

    torch.cuda.set_device(0)
    ctx = arb.default_context(0)
    peaks = load_peaks()
    calibration = measure_alu(ctx)
    ctx.set_autotune(args.autotune)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    wl = args.workload
    cpu_fn = None
    work = None
    if wl == "n32dots":
        case = dot_matmul_n32_p128()
        A, B = arb.Balls.from_raw(case.A[0]), arb.Balls.from_raw(case.B[0])
        C = arb.Balls.empty(32 * 32, 2)

        def step():
            arb.mat_mul(C, A, B, 32, 32, 32, 128, alg=arb.ALG_DOT, ctx=ctx)
        macs, prec, name = 32 ** 3, 128, "real ball matmul N=32 p=128 by dots (exact balls)"
        inbytes, outbytes = A.nbytes() + B.nbytes(), C.nbytes()
        work = dot_work({2: macs}, unique_bytes=3 * 32 * 32 * (8 * 2 + 24))

        def cpu_fn(limit):
            return _oracle_entries(lambda i, j: X.matmul_entry_terms(case.A[0], case.B[0], 32,
                                                                      32, i, j), 32, 32, 32,
                                   128, limit)
    elif wl == "dots":
        bt = batched_dots()
        x, y = arb.Balls.from_raw(bt.x), arb.Balls.from_raw(bt.y)
        res = arb.Balls.empty(len(bt.length), 3)
        t = batch_tensors(bt)
        pmax, lmax = int(bt.prec.max()), int(bt.length.max())

        def step():
            arb.dot(res, x, y, t["xoff"], t["xstep"], t["yoff"], t["ystep"], t["length"],
                    t["prec"], prec_max=pmax, len_max=lmax, ctx=ctx)
        macs, prec = int(bt.length.sum()), 192
        name = bt.name
        inbytes, outbytes = x.nbytes() + y.nbytes(), res.nbytes()
        nd = (bt.prec.astype(np.int64) + 63) // 64
        work = dot_work({int(n): int(bt.length[nd == n].sum()) for n in np.unique(nd)})

        def cpu_fn(limit):
            rng = np.random.default_rng(0)
            done = terms = 0
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < limit:
                b = int(rng.integers(len(bt.length)))
                idx = range(int(bt.xoff[b]), int(bt.xoff[b] + bt.length[b]))
                X.result_exact(X.real_dot_terms(bt.x, idx, bt.y, idx), int(bt.prec[b]), 3)
                done += 1
                terms += int(bt.length[b])
            dt = time.perf_counter() - t0
            return terms / dt, f"{done} dots ({terms} terms) in {dt:.1f} s", dt
    elif wl in ("complex2048", "complex2048_literal"):
        case = complex_matmul_laplace(n=args.complex_n, structured=(wl == "complex2048"))
        n = case.N
        A = [arb.Balls.from_raw(a) for a in case.A]
        B = [arb.Balls.from_raw(b) for b in case.B]
        C = [arb.Balls.empty(n * n, 2), arb.Balls.empty(n * n, 2)]
        # --complex-3m: eq. 2 on both parts truncated under shared thresholds (Section IV-B's
        # omission with Section IV-C's shared scaling)
        mflags = arb.MM_COMPLEX_3M if args.complex_3m else 0
        need = arb.mat_mul_workspace_size(n, n, n, 128, 2, 2, True, arb.ALG_AUTO, mflags)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")

        def step():
            arb.mat_mul(C, A, B, n, n, n, 128, flags=mflags, workspace=ws, ctx=ctx)
        macs, prec = n ** 3, 128
        name = case.name + (", eq. 2 with thresholds shared by both parts (3M)"
                            if args.complex_3m else "")
        inbytes = sum(b.nbytes() for b in A + B)
        outbytes = sum(c.nbytes() for c in C)

        def cpu_fn(limit):
            rng = np.random.default_rng(0)
            done = 0
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < limit:
                i, j = int(rng.integers(n)), int(rng.integers(n))
                re, im = X.complex_dot_terms(case.A, [i * n + k for k in range(n)], case.B,
                                             [k * n + j for k in range(n)])
                X.result_exact(re, 128, 2)
                X.result_exact(im, 128, 2)
                done += 1
            dt = time.perf_counter() - t0
            return done * n / dt, f"{done} complex entries x {n} terms in {dt:.1f} s", dt
    elif wl == "complex2048_uniform":
        # complex N = 2048, p = 128, uniform exponents: the parts' shared scaling fits one block,
        # so --complex-3m takes eq. 2 (three real products) instead of four
        n, prec = 2048, 128
        parts = [matmul_uniform(SEED_BASE + 6 + q, n, prec, -20, 20, rad_bits=120)
                 for q in range(2)]
        cA = [parts[0].A[0], parts[1].A[0]]
        cB = [parts[0].B[0], parts[1].B[0]]
        A = [arb.Balls.from_raw(a) for a in cA]
        B = [arb.Balls.from_raw(b) for b in cB]
        C = [arb.Balls.empty(n * n, 2), arb.Balls.empty(n * n, 2)]
        mflags = arb.MM_COMPLEX_3M if args.complex_3m else 0
        need = arb.mat_mul_workspace_size(n, n, n, prec, 2, 2, True, arb.ALG_AUTO, mflags)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")

        def step():
            arb.mat_mul(C, A, B, n, n, n, prec, flags=mflags, workspace=ws, ctx=ctx)
        macs = n ** 3
        name = (f"complex ball matmul N=2048 p=128, uniform exponents U[-20,20], radii 2^-120 "
                f"relative, {'eq. 2 (3M)' if args.complex_3m else 'four real products (4M)'}")
        inbytes = sum(b.nbytes() for b in A + B)
        outbytes = sum(c.nbytes() for c in C)

        def cpu_fn(limit):
            rng = np.random.default_rng(0)
            done = 0
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < limit:
                i, j = int(rng.integers(n)), int(rng.integers(n))
                re, im = X.complex_dot_terms(cA, [i * n + k for k in range(n)], cB,
                                             [k * n + j for k in range(n)])
                X.result_exact(re, prec, 2)
                X.result_exact(im, prec, 2)
                done += 1
            dt = time.perf_counter() - t0
            return done * n / dt, f"{done} complex entries x {n} terms in {dt:.1f} s", dt
    elif wl == "series":
        # power series exponentials (Section V's dot-product recurrence), many series at once
        from synth import random_balls
        length, batch, prec = 200, 1024, 128
        rng = np.random.default_rng(SEED_BASE + 6)
        raw = random_balls(rng, length * batch, 2, 128, -3, 1, rad_bits=120, rad_zero_frac=0.5)
        a = arb.Balls.from_raw(raw)
        res = arb.Balls.empty(length * batch, 2)
        n = ctypes.c_size_t(0)
        arb._lib.lib().arbgpu_series_exp_workspace_size(ctx.handle, length, batch, prec,
                                                        ctypes.byref(n))
        ws = torch.empty(max(int(n.value), 1), dtype=torch.uint8, device="cuda")

        def step():
            arb.series_exp(res, a, length, batch, prec, workspace=ws, ctx=ctx)
        macs = batch * (length * (length - 1) // 2 + 2 * length)
        work = dot_work({3: macs})  # the working balls carry ceil(p / 64) + 1 limbs
        name = (f"power series exp, {batch} series x {length} coefficients, p={prec}: 128-bit "
                f"mantissas, exponents U[-3,1], radii 2^-120 relative (half zero)")
        inbytes, outbytes = a.nbytes(), res.nbytes()

        def cpu_fn(limit):
            from fractions import Fraction
            from oracle import series as OS
            done = terms = 0
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < limit and done < batch:
                s_ = done
                av = [X.dy_to_fraction(X.mid(raw, k * batch + s_)) for k in range(length)]
                rv = [X.dy_to_fraction(X.rad(raw, k * batch + s_)) for k in range(length)]
                OS.exp_series_radius(av, rv, length)
                done += 1
                terms += length * (length - 1) // 2 + 2 * length
            dt = time.perf_counter() - t0
            return terms / dt, f"{done} series x {length} coefficients in {dt:.1f} s", dt
    else:  # grouped
        cases = grouped_matmuls()
        if args.items:  # a subset of the batch (e.g. one item for a profiler capture)
            cases = [cases[int(t)] for t in args.items.split(",")]
        items = []
        inbytes = outbytes = 0
        for c in cases:
            A, B = arb.Balls.from_raw(c.A[0]), arb.Balls.from_raw(c.B[0])
            Cc = arb.Balls.empty(c.N * c.N, (c.prec + 63) // 64)
            items.append(dict(C=Cc, A=A, B=B, M=c.M, K=c.K, N=c.N, prec=c.prec))
            inbytes += A.nbytes() + B.nbytes()
            outbytes += Cc.nbytes()

        def step():
            arb.mat_mul_batched(items, ctx=ctx)
        macs = sum(c.M * c.K * c.N for c in cases)
        prec = 1024
        name = ("grouped batch of 256 real ball matmuls, N U[16,512], p in {64..1024}, "
                "exponents U[-50,50], radii 2^-(p-8)")
        if args.items:
            name = f"items {args.items} of the " + name

        def cpu_fn(limit):
            rng = np.random.default_rng(0)
            done = terms = 0
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < limit:
                c = cases[int(rng.integers(len(cases)))]
                i, j = int(rng.integers(c.N)), int(rng.integers(c.N))
                X.result_exact(X.matmul_entry_terms(c.A[0], c.B[0], c.K, c.N, i, j), c.prec,
                               (c.prec + 63) // 64)
                done += 1
                terms += c.K
            dt = time.perf_counter() - t0
            return terms / dt, f"{done} entries of random items ({terms} terms) in {dt:.1f} s", dt
    for _ in range(args.warmup):
        step()
    ctx.check()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    l0 = ctx.launch_count()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    clocks = sampler.stop()
    ctx.check()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    value = macs * args.steps / (ms * 1e-3) / 1e9
    # the per-kernel breakdown from the library's event trace, in a separate pass of the same
    # steps (the events around every launch stay out of the timed region)
    ctx.trace(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        flush.zero_()
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    recs = ctx.trace_read(max_entries=1 << 18)
    ctx.trace(False)
    ctx.check()
    kernels = kernel_summary(recs, t0.elapsed_time(t1))
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roofline = None
    if kernels:
        dom = max(kernels.items(), key=lambda kv: kv[1]["ms_total"])
        if dom[0] in DOT_KERNELS and work is not None:
            roofline = dot_roofline(kernels, work, args.steps, peaks, sm_mhz)
            roofline["share_of_step"] = round(sum(
                kernels.get(k, {}).get("share", 0) or 0 for k in DOT_KERNELS), 4)
        else:
            roofline = roofline_of(dom[0], dom[1], peaks, sm_mhz, limb_n=(prec + 63) // 64)
            roofline["share_of_step"] = dom[1]["share"]
    graph = None
    if wl == "n32dots":
        # latency of the call replayed from a CUDA graph (no host work between calls)
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        with torch.cuda.graph(g):
            step()
        g.replay()
        torch.cuda.synchronize()
        reps = 200
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record()
        for _ in range(reps):
            g.replay()
        gb.record()
        torch.cuda.synchronize()
        gus = ga.elapsed_time(gb) * 1e3 / reps
        graph = {"us_per_call": gus, "GMAC_s": macs / (gus * 1e-6) / 1e9, "calls": reps,
                 "l2": "not flushed between replays (the inputs stay in L2)"}
        ctx.check()
    r, sample, _dt = cpu_fn(args.cpu_seconds)
    line = {"metric": "ball multiply-adds per second (complex MACs for complex)",
            "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64 limbs / exact integer products",
            "data": "synthetic", "config": {"workload": name, "l2": "flushed before every step"},
            "gpu_launches": launches, "roofline": roofline, "kernels": kernels,
            "cpu_baseline": {"value": r / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "io_bytes": {"in": inbytes, "out": outbytes}, "clocks": clocks,
            "calibration": calibration, "autotune": dict(ctx.autotune_stats(), on=args.autotune,
                                                        algorithm=ctx.autotune_alg_stats())}
    if graph:
        line["us_per_call"] = ms / args.steps * 1e3
        line["graph_replay"] = graph
    print(json.dumps(line), flush=True)


def _oracle_entries(terms_of, M, K, N, prec, limit):
    import numpy as np
    from oracle import exact as X
    rng = np.random.default_rng(0)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < limit:
        i, j = int(rng.integers(M)), int(rng.integers(N))
        X.result_exact(terms_of(i, j), prec, (prec + 63) // 64)
        done += 1
    dt = time.perf_counter() - t0
    return done * K / dt, f"{done} entries x {K} terms in {dt:.1f} s", dt


# --------------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", type=int, default=256)
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--alg", default="auto", choices=["auto", "dot", "block"])
    ap.add_argument("--no-compare", action="store_true", help="skip the p=128 / dot-path lines")
    ap.add_argument("--ref-entries", type=int, default=48)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--complex-3m", action="store_true",
                    help="complex workloads: the complex product by eq. 2 (three real products)")
    ap.add_argument("--complex-n", type=int, default=2048,
                    help="complex2048 / complex2048_literal: the matrix size (2048: the workload; "
                         "smaller for profiling captures)")
    ap.add_argument("--autotune", action="store_true",
                    help="turn on the library's engine autotuner (the warm-up steps decide)")
    ap.add_argument("--items", default="",
                    help="grouped workload only: comma-separated item indices to run instead of "
                         "the whole batch")
    ap.add_argument("--workload", default="n512",
                    choices=["n512", "n32dots", "dots", "complex2048", "complex2048_literal",
                             "complex2048_uniform", "series", "grouped"],
                    help="n512 (default): the headline; the others are the remaining synthetic "
                         "workloads, one JSON line each")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "n512":
        run_workload(args)
        return

    import torch
    import torch.distributed as dist

    import paper_1901_04289_gb300 as arb
    from synth.workloads import block_matmul_n512, matmul_uniform

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    ctx = arb.default_context(local)
    peaks = load_peaks()
    calibration = measure_alu(ctx)
    ctx.set_autotune(args.autotune)
    algs = {"auto": arb.ALG_AUTO, "dot": arb.ALG_DOT, "block": arb.ALG_BLOCK}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def make(prec):
        if args.n == N_DEFAULT:
            return block_matmul_n512(prec=prec)
        return matmul_uniform(1901042893, args.n, prec, -20, 20, rad_bits=250)

    def timed(case, prec, alg, steps, warmup, e2e=False, trace=False):
        n = case.N
        nl = (prec + 63) // 64
        A = arb.Balls.from_raw(case.A[0], device=dev)
        B = arb.Balls.from_raw(case.B[0], device=dev)
        C = arb.Balls.empty(case.M * n, nl, device=dev)
        hA = hB = hC = None
        if e2e:
            hA = arb.Balls.from_raw(case.A[0], pin=True)
            hB = arb.Balls.from_raw(case.B[0], pin=True)
            hC = arb.Balls(*(torch.empty_like(t, device="cpu").pin_memory() for t in C.tensors()))
        need = arb.mat_mul_workspace_size(case.M, case.K, n, prec, A.nlimbs, B.nlimbs, False, alg)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)

        def step():
            if e2e:
                A.copy_from_(hA, non_blocking=True)
                B.copy_from_(hB, non_blocking=True)
            arb.mat_mul(C, A, B, case.M, case.K, n, prec, alg=alg, workspace=ws, ctx=ctx)
            if e2e:
                hC.copy_from_(C, non_blocking=True)

        for _ in range(warmup):
            step()
        ctx.check()
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = ctx.launch_count()
        if trace:
            ctx.trace(True)
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        launches = ctx.launch_count() - l0
        recs = ctx.trace_read(max_entries=1 << 18) if trace else []
        ctx.trace(False)
        ctx.check()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        h2d = (A.nbytes() + B.nbytes()) if e2e else 0
        d2h = C.nbytes() if e2e else 0
        return ms, launches, recs, h2d, d2h

    def timed_e2e(case, prec, alg, steps, warmup):
        """End to end through the public call: every step copies its inputs from pinned host
        memory, multiplies, and reads the product back.  Steps are pipelined over three streams
        with two device buffers each (the copies of step k + 1, queued before the product of step
        k, and the read-back of step k - 1 overlap the product of step k); the time is the span
        from the first copy to the last read-back."""
        n = case.N
        nl = (prec + 63) // 64
        # every ball array is one packed buffer, so each moves in one copy
        Ad = [arb.Balls.from_raw(case.A[0], device=dev, packed=True) for _ in range(2)]
        Bd = [arb.Balls.from_raw(case.B[0], device=dev, packed=True) for _ in range(2)]
        Cd = [arb.Balls.packed(case.M * n, nl, device=dev) for _ in range(2)]
        hA = arb.Balls.from_raw(case.A[0], pin=True, packed=True)
        hB = arb.Balls.from_raw(case.B[0], pin=True, packed=True)
        hC = [arb.Balls.packed(case.M * n, nl, pin=True) for _ in range(2)]
        need = arb.mat_mul_workspace_size(case.M, case.K, n, prec, Ad[0].nlimbs, Bd[0].nlimbs,
                                          False, alg)
        ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
        s_in, s_mm, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

        def run(count):
            ev = lambda: torch.cuda.Event()
            h2d, mm, d2h = [], [], []

            def copy_in(k):  # the inputs of step k into buffer k mod 2
                with torch.cuda.stream(s_in):
                    if k >= 2:
                        s_in.wait_event(mm[k - 2])  # the product of step k - 2 read that buffer
                    Ad[k % 2].copy_from_(hA, non_blocking=True)
                    Bd[k % 2].copy_from_(hB, non_blocking=True)
                    h2d.append(ev())
                    h2d[k].record(s_in)

            if count:
                copy_in(0)
            for k in range(count):
                b = k % 2
                if k + 1 < count:
                    copy_in(k + 1)  # queued before step k's product, so it runs beside it
                with torch.cuda.stream(s_mm):
                    s_mm.wait_event(h2d[k])
                    if k >= 2:
                        s_mm.wait_event(d2h[k - 2])  # step k - 2's result has been read back
                    arb.mat_mul(Cd[b], Ad[b], Bd[b], case.M, case.K, n, prec, alg=alg,
                                workspace=ws, ctx=ctx, stream=s_mm)
                    mm.append(ev())
                    mm[k].record(s_mm)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(mm[k])
                    hC[b].copy_from_(Cd[b], non_blocking=True)
                    d2h.append(ev())
                    d2h[k].record(s_out)

        run(warmup)
        torch.cuda.synchronize()
        ctx.check()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0.record(s_in)
        run(steps)
        s_out.wait_stream(s_in)
        s_out.wait_stream(s_mm)
        t1.record(s_out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ctx.check()
        return (t0.elapsed_time(t1), hA.buffer.numel() + hB.buffer.numel(),
                hC[0].buffer.numel())

    prec = args.prec
    alg = algs[args.alg]
    case = make(prec)
    macs = case.M * case.K * case.N
    ctx.reserve(prec, case.K)  # the multimodular tables, uploaded before any timing
    sampler = ClockSampler(local)
    sampler.start()
    ms, launches, _, _, _ = timed(case, prec, alg, args.steps, args.warmup)
    # the timed steps last milliseconds and the sampler reads every 200 ms: keep the same steps
    # running for a second more so that the clock record covers this load
    soak = max(1, int(1000.0 / max(ms / args.steps, 1e-3)))
    timed(case, prec, alg, min(soak, 20000), 0)
    clocks = sampler.stop()
    if clocks:
        clocks["window"] = "the timed steps and 1 s of the same steps right after them"
    # the per-kernel breakdown from the library's event trace, in a separate pass (the events
    # around every launch stay out of the timed region)
    ms_traced, _, recs, _, _ = timed(case, prec, alg, args.steps, 1, trace=True)
    ms_max, value = replica_throughput(ms, macs * args.steps, world, dev)
    # the end-to-end pipeline fills (the first upload) and drains (the last product and read-back)
    # once per timed region: over E2E_MIN_STEPS steps or more, its rate is the streaming one
    e2e_steps = max(args.steps, E2E_MIN_STEPS)
    e2e_ms, h2d, d2h = timed_e2e(case, prec, alg, e2e_steps, 3)
    e2e_value = macs * e2e_steps / (e2e_ms * 1e-3) / 1e9

    # roofline of the dominant kernel (and of the tensor-core kernel), from the library's
    # per-launch events
    kernels = kernel_summary(recs, ms_traced)
    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roofline = None
    tensor = None
    if kernels:
        dom = max(kernels.items(), key=lambda kv: kv[1]["ms_total"])
        if dom[0] in DOT_KERNELS:
            n = (prec + 63) // 64
            ent = (case.M * case.K + case.K * case.N + case.M * case.N) * (8 * n + 24)
            roofline = dot_roofline(kernels, dot_work({n: macs}, unique_bytes=ent), args.steps,
                                    peaks, sm_mhz)
            roofline["share_of_step"] = round(sum(
                kernels.get(k, {}).get("share", 0) or 0 for k in DOT_KERNELS), 4)
        else:
            roofline = roofline_of(dom[0], dom[1], peaks, sm_mhz)
            roofline["share_of_step"] = dom[1]["share"]
        for tn in ("crt_gemm", "digit_gemm_mid"):
            if tn in kernels:
                tensor = roofline_of(tn, kernels[tn], peaks, sm_mhz)
                tensor["share_of_step"] = kernels[tn]["share"]
                break
        if args.n == N_DEFAULT and prec == 256 and args.alg == "auto":
            for r in (roofline, tensor):
                if r and r.get("kernel") in TRAFFIC_N512_P256:
                    r["traffic"] = TRAFFIC_N512_P256[r["kernel"]]
                    r["traffic_source"] = "ncu capture, profiles/multimodular_n512_p256_full.md"

    compare = {}
    if not args.no_compare and args.n == N_DEFAULT:
        for p in (128, 256):
            c = case if p == prec else make(p)
            for nm, a in (("auto", arb.ALG_AUTO), ("dot", arb.ALG_DOT)):
                if p == prec and a == alg:
                    compare[f"{nm}_p{p}"] = value / world
                    continue
                t, _, _, _, _ = timed(c, p, a, 3, 1)
                compare[f"{nm}_p{p}"] = c.M * c.K * c.N * 3 / (t * 1e-3) / 1e9
        for p in (128, 256):
            compare[f"speedup_vs_dot_p{p}"] = compare[f"auto_p{p}"] / compare[f"dot_p{p}"]

    cpu = None
    if rank == 0 and world == 1:
        import multiprocessing as mp
        cores = host_cores()
        with mp.get_context("spawn").Pool(cores) as pool:
            r, n_ent, dt = oracle_all_cores(prec, case.N, args.cpu_seconds, pool, cores)
        cpu = {"value": r / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_ent} random output entries x {case.K} terms, {cores} processes "
                         f"for {dt:.1f} s each (exact Python-integer dot, one rounding)"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64 limbs / exact integer products", "data": "synthetic",
                "config": {"workload": workload_name(case.N, prec), "alg": args.alg,
                           "l2": "flushed (512 MiB write) before every timed step",
                           "parallelism": f"replicas x{world}"},
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h,
                        "steps": e2e_steps,
                        "how": "every step copies A, B from pinned host memory and reads C back "
                               "(one packed buffer per ball array); steps pipelined over 3 "
                               "streams x 2 buffers, no L2 flush; the span from the first "
                               "upload to the last read-back over `steps` steps"},
                "gpu_launches": launches, "roofline": roofline, "tensor_core": tensor,
                "kernels": kernels,
                "cpu_baseline": cpu,
                "clocks": clocks, "compare": compare, "peaks_source": peaks["_source"],
                "calibration": calibration,
                "autotune": dict(ctx.autotune_stats(), on=args.autotune,
                                 algorithm=ctx.autotune_alg_stats())}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
