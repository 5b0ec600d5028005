"""Host-side logic of bench.py (CPU): the roofline arithmetic, the kernel-share table and the
reference arm's JSON line."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6792.4, "sm_max_mhz": 2070.0}


def _prof():
    # per-kernel totals as ch_profile_read reports them: summed ms, launches, algorithmic bytes, FMAs
    return {
        "cheb_step_f64": {"ms": 130.0, "launches": 7500, "bytes": 7500 * 37.2e6, "fmas": 7500 * 4.73e6},
        "cheb_step_coarse_f64": {"ms": 55.0, "launches": 5200, "bytes": 5200 * 2.0e6, "fmas": 5200 * 0.25e6},
        "restrict_f32": {"ms": 10.0, "launches": 800, "bytes": 800 * 9.0e6, "fmas": 800 * 0.5e6},
    }


def test_roofline_of_an_alu_bound_fp64_kernel():
    """The dominant kernel is the one with the largest summed time; an FP64 kernel above the
    FMA-per-byte balance point is rated against the derived FP64 peak
    (152 SMs x 2 FMA/clk x 2 flop x max clock)."""
    r = bench.roofline(_prof(), PEAKS)
    assert r["kernel"] == "cheb_step_f64" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = 152 * 2 * 2 * 2070e6 / 1e12
    per_launch_s = 130.0 / 7500 * 1e-3
    achieved = 2 * 4.73e6 / per_launch_s / 1e12
    assert math.isclose(r["peak"], peak, rel_tol=1e-12)
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(r["frac"], achieved / peak, rel_tol=1e-12)
    assert math.isclose(r["share_of_kernel_time"], 130.0 / 195.0, rel_tol=1e-12)
    assert math.isclose(r["algorithmic_bytes_per_launch"], 37.2e6, rel_tol=1e-12)
    committed = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    assert r["traffic"] == committed["cheb_step_f64"]["bytes_per_launch"]  # the ncu figure committed for this kernel


def test_roofline_of_an_hbm_bound_kernel():
    """An FP32 kernel is rated against the measured HBM copy bandwidth."""
    prof = {"cheb_step_f32": {"ms": 50.0, "launches": 7000, "bytes": 7000 * 18.6e6, "fmas": 7000 * 4.73e6},
            "orth_dots_f64": {"ms": 5.0, "launches": 160, "bytes": 160 * 40e6, "fmas": 160 * 3e6}}
    r = bench.roofline(prof, PEAKS)
    assert r["kernel"] == "cheb_step_f32" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    achieved = 18.6e6 / (50.0 / 7000 * 1e-3) / 1e9
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-12)
    assert math.isclose(r["frac"], achieved / 6792.4, rel_tol=1e-12)
    assert r["peak_source"].startswith("measured")
    r_fallback = bench.roofline(prof, {})
    assert r_fallback["peak"] == 6800.0 and r_fallback["peak_source"] == "fallback"


def test_roofline_takes_the_in_sequence_launch_time():
    """With the kernel timed in sequence (back-to-back launches in one graph) the launch time is
    that one, the event-timed figures are kept beside it, and a rate above the HBM peak (an
    L2-resident working set) carries the note that says so; another dominant kernel ignores it."""
    prof = {"cheb_step_f32": {"ms": 50.0, "launches": 7000, "bytes": 7000 * 18.6e6, "fmas": 7000 * 4.73e6}}
    seq = {"avg_launch_us": 2.4, "achieved_GBps": 7750.0}
    r = bench.roofline(prof, PEAKS, seq)
    achieved = 18.6e6 / 2.4e-6 / 1e9
    assert math.isclose(r["achieved"], achieved, rel_tol=1e-12) and r["avg_launch_us"] == 2.4
    assert math.isclose(r["event_timed"]["avg_launch_us"], 1e3 * 50.0 / 7000, rel_tol=1e-12)
    assert r["in_sequence"] is seq and r["frac"] > 1.0 and "L2" in r["note"]
    r64 = bench.roofline(_prof(), PEAKS, {"avg_launch_us": 11.76})
    assert r64["bound"] == "alu"
    assert math.isclose(r64["achieved"], 2 * 4.73e6 / 11.76e-6 / 1e12, rel_tol=1e-12)
    other = {"orth_dots_f64": {"ms": 5.0, "launches": 160, "bytes": 160 * 40e6, "fmas": 160 * 3e6}}
    r_other = bench.roofline(other, PEAKS, seq)
    assert "in_sequence" not in r_other and math.isclose(r_other["avg_launch_us"], 1e3 * 5.0 / 160)


def test_top_kernels_are_sorted_shares():
    t = bench.top_kernels(_prof())
    names = list(t)
    assert names == ["cheb_step_f64", "cheb_step_coarse_f64", "restrict_f32"]
    assert math.isclose(sum(v["share"] for v in t.values()), 1.0, rel_tol=1e-12)
    assert math.isclose(t["restrict_f32"]["GBps"], 9.0e6 / (10.0 / 800 * 1e-3) / 1e9, rel_tol=1e-12)


def test_reference_arm_line():
    """`--impl reference` times the oracle (the CPU program standing in for the reference) and
    prints the contract's line with the warm-up steps it actually ran."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--nx", "16", "--ny", "16", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 3
    for key in ("metric", "value", "unit", "n_gpus", "ms_per_step", "higher_is_better", "scaling",
                "dtype", "data", "config"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert "3 untimed and 2 timed steps" in line["cpu_baseline"]["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
