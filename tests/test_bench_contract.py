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
    assert bench.ops_per_attempt(g, "philox") == pytest.approx(ops + 3)


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
