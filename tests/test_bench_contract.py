"""bench.py's roofline arithmetic on the CPU: the fraction it reports is the
algorithmic work per second over the stated peak."""
from __future__ import annotations

import json
import os

import pytest

import bench
from paper_1004_0024_gb300 import workloads as W


def test_alu_roofline_counts_algorithmic_ops_over_the_issue_peak():
    c = W.config1()
    g = c["graph"]
    attempts = g.n * c["R"] * 200
    r = bench.roofline(c, "mt19937", attempts, 36.0, 1, {"sm_mhz": 2000.0}, 2)
    ops = 17 + 6 + 3 * float(g.row_ptr[-1]) / g.n
    assert r["bound"] == "alu" and r["ops_per_attempt"] == pytest.approx(ops)
    assert r["achieved"] == pytest.approx(attempts * ops / 0.036 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] is None  # lean kernel (variant 2): no DRAM capture of its current build
    assert bench.ops_per_attempt(g, "philox") == pytest.approx(ops + 3)


def test_measured_traffic_of_the_packed_kernel_scales_with_the_sweeps():
    """The packed kernel's DRAM bytes come from its 1-pass ncu captures: the
    200-sweep launch as captured, other launch lengths on the line through the
    10- and 200-sweep captures; other kernels and generators report none."""
    c = W.config1()
    g = c["graph"]
    per_sweep = g.n * c["R"]
    r = bench.roofline(c, "mt19937", per_sweep * 200, 19.2, 1, {"sm_mhz": 2070.0}, 4)
    assert r["traffic"] == pytest.approx(3311.4e6)
    r10 = bench.roofline(c, "mt19937", per_sweep * 20, 2.3, 2, {"sm_mhz": 2070.0}, 4)
    assert r10["traffic"] == pytest.approx(234.3e6)
    assert "ncu" in r["traffic_basis"]
    assert bench.roofline(c, "philox", per_sweep * 200, 19.6, 1, {"sm_mhz": 2070.0}, 4)["traffic"] is None


def test_hbm_roofline_of_streamed_words():
    c = W.config3()
    g = c["graph"]
    sweeps, launches = 500, 63
    attempts = g.n * c["R"] * sweeps
    r = bench.roofline(c, "mt19937", attempts, 1000.0, launches, None, 2, name="cfg3")
    bpa = 4.0 + 6.0 / (sweeps / launches)
    peak = json.load(open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    assert r["bound"] == "hbm" and r["bytes_per_attempt"] == pytest.approx(bpa)
    assert r["achieved"] == pytest.approx(attempts * bpa / 1.0 / 1e9)
    assert r["peak"] == pytest.approx(float(peak)) and r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_cpu_baseline_uses_the_workloads_split_couplings(monkeypatch):
    """The oracle leg times the same chain the GPU runs: with split couplings
    (cfg1-trotter) it sets the workload's K; a bounded sample of a small
    layered model runs in a fraction of a second here."""
    import numpy as np

    import oracle
    seen = []
    orig = oracle.Sim.set_trotter

    def spy(self, K):
        seen.append(np.asarray(K).copy())
        return orig(self, K)

    monkeypatch.setattr(oracle.Sim, "set_trotter", spy)
    c = dict(W.config0(), R=4, betas=W.geometric_betas(4, 0.1, 3.0))
    c["K"] = W.trotter_couplings(c["betas"], 2.0, 16)
    r = bench.cpu_baseline(c, "philox", 0.05)
    assert len(seen) == 1 and np.array_equal(seen[0], c["K"])
    assert r["kind"] == "oracle" and r["unit"] == "attempts/s" and r["value"] > 0
    assert bench.workload("cfg1-trotter")["K"].shape == (256,)
    assert "split couplings" in bench.WORKLOAD_NAMES["cfg1-trotter"]


def test_throttled_or_clock_locked_runs_are_remeasured():
    """Rejected: hw / thermal slowdown, or an SM clock well below its maximum
    with no reason active; kept: the power cap, full clocks, no samples."""
    base = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(base)
    assert not bench.clocks_rejected(None)
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(base, reasons=[r]))
    assert not bench.clocks_rejected(dict(base, sm_mhz=1500.0, reasons=["sw_power_cap"]))
    assert bench.clocks_rejected(dict(base, sm_mhz=1100.0))
    assert bench.any_rank(True, 1) and not bench.any_rank(False, 1)


def test_clock_samples_and_the_remeasure_rule(tmp_path):
    """nvidia-smi's CSV rows (no header, no units) give the median SM clock,
    the maximum and the active throttle reasons; a timed region is measured
    again after a hardware or thermal slowdown, or with the SM clock well
    below its maximum and no reason given, but not for sw_power_cap alone."""
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1900, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc, s.path = Done(), str(path)
    c = s.stop()
    assert c == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()
    assert not bench.clocks_rejected(c)
    assert not bench.clocks_rejected(None)
    assert bench.clocks_rejected({"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown"]})
    assert bench.clocks_rejected({"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": ["sw_thermal_slowdown"]})
    assert bench.clocks_rejected({"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": []})
    assert not bench.clocks_rejected({"sm_mhz": 1200.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"]})


def test_latency_floor_is_levels_times_the_level_chain():
    import bench
    bench._LATENCIES = {"shared_load": 30.0, "int_mad": 4.0, "shuffle": 36.0, "barrier_8_warps": 24.0}
    try:
        f = bench.latency_floor(400, 200, 26.0, {"sm_mhz": 2000.0})
    finally:
        bench._LATENCIES = None
    cyc = 30.0 + bench.LEVEL_CHAIN_INT_OPS * 4.0 + 36.0 + 24.0
    assert f["cycles_per_level"] == cyc
    assert abs(f["ms_per_launch"] - 400 * 200 * cyc / 2.0e6) < 1e-9
    assert abs(f["frac"] - f["ms_per_launch"] / 26.0) < 1e-12



def test_latency_floor_only_for_resident_ladders():
    f = bench.latency_floor(83, 500, 1086.0, {"sm_mhz": 2070.0}, resident=0)
    assert f["frac"] is None and "resident" in f["why"]
