"""Host-side pieces of bench.py that need no GPU: the clock-sample summary, the workload
config both arms print, and the source hash that guards the committed DRAM traffic."""
import json
import os

import bench


def test_clock_summary_flags_throttling():
    ok = ["0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"] * 3
    s = bench.Clocks.summarise(ok + ["garbage line\n"])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == [] and s["samples"] == 3
    hot = ["0, 1500, 2070, 1390.0, 0x04, Not Active, Not Active, Not Active, Active\n",
           "0, 1400, 2070, 1395.0, 0x48, Active, Not Active, Not Active, Active\n",
           "0, 1600, 2070, 1380.0, 0x00, Not Active, Not Active, Not Active, Not Active\n"]
    s = bench.Clocks.summarise(hot)
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.Clocks.summarise([])["reasons"] == ["no samples"]


def test_both_arms_name_the_same_workload():
    c = bench.workload_config(1)
    assert c["workload"] == bench.WL.name and c["grid"] == list(bench.WL.shape)
    assert c["ntraj_per_gpu"] == bench.WL.ntraj and "trajectories sharded over 1" in c["parallelism"]
    json.dumps(c)


def test_traffic_figures_follow_the_sources():
    """The committed ncu DRAM bytes are reported only while the pass sources hash to the
    value stored beside them."""
    p = os.path.join(bench.ROOT, "profiles", "dram_traffic.json")
    d = json.load(open(p))
    assert set(d["per_launch_bytes"]) == {"xpass", "strided_pass"}
    if d["source_hash"] == bench.kernel_source_hash():
        assert bench.ncu_traffic("xpass") == float(d["per_launch_bytes"]["xpass"])
    else:
        assert bench.ncu_traffic("xpass") is None


def test_step_stats_median_and_spread():
    s = bench.step_stats([10.0, 12.0, 11.0, 30.0, 11.5])
    assert s["n"] == 5 and s["median_ms"] == 11.5 and s["min_ms"] == 10.0 and s["max_ms"] == 30.0
    assert abs(s["spread_pct"] - 100.0 * 20.0 / 11.5) < 1e-12
    assert s["p10_ms"] == 10.0 and s["p90_ms"] == 30.0
    assert bench.step_stats([]) is None
