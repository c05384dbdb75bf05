"""Host-side logic of bench.py, on the CPU: the roofline arithmetic (achieved = algorithmic work per
launch / average launch time, frac = achieved / peak), the per-kernel trace summary, the dot path's
choice of its binding resource, and the reference arm's JSON line (the oracle timed on a bounded
sample)."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_summary_adds_launches_and_shares():
    recs = [("crt_gemm", 0.05, 100), ("residues", 0.02, 7), ("crt_gemm", 0.05, 100)]
    s = bench.kernel_summary(recs, 0.2)
    assert s["crt_gemm"] == {"launches": 2, "ms_total": 0.1, "share": 0.5, "units": 200}
    assert s["residues"]["launches"] == 1 and s["residues"]["share"] == pytest.approx(0.1)


def test_tensor_roofline_counts_two_flops_per_digit_mac():
    # ten launches of 1e11 digit MACs in 0.5 ms: 50 us each -> 2e11 flops / 5e-5 s = 4 PFLOP/s
    k = {"ms_total": 0.5, "launches": 10, "units": 10 * 10 ** 11}
    r = bench.roofline_of("crt_gemm", k, {"bf16_tflops": 2000.0}, 2070.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4000.0)
    assert r["frac"] == pytest.approx(2.0)


def test_residue_roofline_is_algorithmic_bytes_over_time():
    k = {"ms_total": 0.5, "launches": 10, "units": 10 * 10 ** 8}  # 1e8 bytes per 50 us launch
    r = bench.roofline_of("residues", k, {"hbm_gbs": 8000.0}, 2070.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["frac"] == pytest.approx(0.25)


def test_alu_peak_is_derived_from_units_and_clock():
    k = {"ms_total": 1.0, "launches": 1, "units": 10 ** 9}
    r = bench.roofline_of("block_round", k, {}, 1000.0)
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(bench.SMS * bench.IMAD_PER_CLK_PER_SM * 1e9 / 1e12)
    assert r["achieved"] == pytest.approx(1.0)  # 1e9 multiply-adds in 1 ms


def test_dot_work_closed_forms():
    w = bench.dot_work({2: 100, 1: 10})
    assert w["terms"] == 110
    assert w["mults"] == 4 * 4 * 100 + 4 * 1 * 10
    assert w["bytes"] == 2 * (16 + 24) * 100 + 2 * (8 + 24) * 10
    assert bench.dot_work({3: 5}, unique_bytes=123)["bytes"] == 123


def test_dot_roofline_takes_the_slower_resource():
    peaks = {"hbm_gbs": 1000.0}
    kern = {"dot_fused": {"ms_total": 2.0, "launches": 2}}
    # bytes-heavy: 1e9 bytes take 1 ms at 1 TB/s, 1e6 multiplies almost nothing
    r = bench.dot_roofline(kern, {"terms": 1, "mults": 10 ** 6, "bytes": 10 ** 9}, 2, peaks, 2070.0)
    assert r["bound"] == "hbm"
    assert r["achieved"] == pytest.approx(10 ** 9 / 1e-3 / 1e9)  # one call per ms
    # multiply-heavy
    r = bench.dot_roofline(kern, {"terms": 1, "mults": 10 ** 13, "bytes": 10}, 2, peaks, 2070.0)
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(10 ** 13 / 1e-3 / 1e12)


def test_reference_arm_prints_one_oracle_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
         "--warmup", "0", "--ref-entries", "2"],
        capture_output=True, text=True, timeout=300, cwd=ROOT,
        env={**os.environ, "RANK": "0"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "N=512 p=256" in d["config"]["workload"]
