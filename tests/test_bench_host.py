"""Host logic of bench.py (CPU only): the clock summary that decides whether a timed run counts,
and the gate that reports recorded DRAM traffic only while the kernel sources are unchanged."""
import hashlib
import json
import os
import shutil

import bench


def _line(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {smax}, 512.3, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}\n"


def test_clock_summary_median_max_and_reasons():
    lines = [_line(2070, 2070), _line(1995, 2070, cap="Active"), _line(2070, 2070),
             "garbage line\n", "0, [N/A], 2070, 1, 0, Not Active, Not Active, Not Active, Not Active\n"]
    got = bench.summarise_clocks(lines)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_summary_reports_every_throttle_reason():
    lines = [_line(1500, 2070, hw="Active"), _line(1400, 2070, hwt="Active"), _line(1300, 2070, swt="Active"),
             _line(1200, 2070)]
    got = bench.summarise_clocks(lines)
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert got["sm_mhz"] == 1350.0 and got["samples"] == 4


def test_clock_summary_without_samples_is_none():
    assert bench.summarise_clocks([]) is None
    assert bench.summarise_clocks(["0, N/A\n"]) is None


def test_recorded_traffic_is_dropped_when_a_kernel_source_changes(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "roofline_traffic.json")))
    h = hashlib.sha256()
    for f in rec["source_files"]:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copyfile(os.path.join(bench.ROOT, f), dst)
        h.update(dst.read_bytes())
    rec["source_sha256"] = h.hexdigest()   # a record taken on exactly these sources
    (tmp_path / "profiles").mkdir(exist_ok=True)
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.recorded_traffic()
    assert got is not None and got["kernels"] == rec["kernels"]
    src = tmp_path / rec["source_files"][0]
    src.write_bytes(src.read_bytes() + b"\n")
    assert bench.recorded_traffic() is None


def test_one_thread_oracle_leg_runs_in_a_child_process():
    from synthetic import HEAT2D_K2_N16_Q2 as w
    got = bench.cpu_baseline_one_thread(w, timeout_s=120)
    assert "error" not in got, got
    assert got["cores"] == 1 and got["value"] > 0 and got["unit"] == bench.UNIT


def test_smoother_alu_side_of_the_roofline():
    from synthetic import HEAT3D_K4_N32_Q3 as w
    r = bench.smoother_alu(w, 3, 0.069)
    # 32^3 cells x (14 5^4 + 4 5^3) flops x 3 blocks, + (5 x 6 + 1) / 6 flops x 3 x 2,048,383
    flops = 32 ** 3 * 9250 * 3 + 31 / 6 * 3 * 2_048_383
    assert abs(r["flops_per_launch"] - flops) < 1e-6 * flops
    assert abs(r["achieved"] - flops / 0.069e-3 / 1e12) < 1e-9
    assert abs(r["peak"] - 152 * 128 * 2.07e9 * 2 / 1e12) < 1e-9 and 0 < r["frac"] < 1


def test_oracle_replicas_use_every_process():
    """The CPU baseline runs one single-threaded oracle replica per process and reports whole-host
    throughput: two replicas of a tiny problem report twice the units of one over the slowest time."""
    import bench
    from synthetic import Workload
    w = Workload("tiny", 3, 2, 4, 2, 1e-2, 1)
    value, nproc, per = bench.oracle_replicas(w, steps=2, nproc=2, timeout_s=120)
    assert nproc in (1, 2) and per > 0
    assert abs(value - nproc * w.Q * w.n_interior / per) <= 1e-9 * value
