"""Host-side pieces of bench.py that need no GPU: the CPU-oracle baseline on a
small copy of the deblurring workload, with all threads and with one."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_sample_scales_its_phases_to_the_solve():
    w = bench.WL.scaled(bench.WL.DEBLUR512, 48, ell=6)
    r = bench.oracle_sample(w, 7)
    ph = r["phase_s"]
    total = w.ell * ph["col"] + ph["factor"] + 50 * ph["power"] + 7 * ph["iteration"]
    assert r["kind"] == "oracle" and r["unit"] == "ms" and r["cores"] >= 1
    # phases are rounded to the millisecond in the report
    assert abs(r["value"] - 1e3 * total) <= 1e3 * (w.ell + 1 + 50 + 7) * 5e-4 + 0.1
    json.dumps(r)


def test_one_thread_sample_runs_in_its_own_interpreter():
    w = bench.WL.scaled(bench.WL.DEBLUR512, 48, ell=6)
    r = bench.oracle_sample_one_thread(w, 7)
    assert "error" not in r, r
    assert r["cores"] == 1 and r["value"] > 0 and "48x48" in r["sample"]


def test_step_stats():
    s = bench.step_stats([3.0, 1.0, 2.0, 10.0])
    assert s == {"mean": 4.0, "median": 2.5, "best": 1.0, "n": 4}


def test_clock_log_summary(tmp_path):
    p = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1300.2, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    p.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler.summarise(str(p))
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    # without nvidia-smi (or before start) the sampler reports itself unavailable
    c = bench.ClockSampler(0, str(tmp_path))
    assert c.path.startswith(str(tmp_path))
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_dual_stop_report():
    # skipped steps per timed solve against the steps the solve issues
    # (n_inner per WAPG iteration)
    w = bench.WL.PRESETS["ct512_parallel_tv_f32"]
    r = bench.dual_stop_info(w, 31850.0, 1774, 81067.0, 4504)
    assert r["precond"]["of"] == 1774 * w.n_inner and r["plain"]["of"] == 4504 * w.n_inner
    assert r["precond"]["fraction"] == round(31850.0 / (1774 * w.n_inner), 4)
    assert 0.0 <= r["plain"]["fraction"] <= 1.0
    json.dumps(r)
