"""Failure detection without a GPU fault (GPU): bounded waits that are made to
run out report ISING_ERR_TIMEOUT and leave the context usable; an allocation
cap stands in for device memory running out."""
import numpy as np
import pytest

import oracle
from paper_1004_0024_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1004_0024_gb300 import ising as mod
    return mod


def _still_works(ising):
    c = W.config0()
    dev = ising.Ising(c["graph"], c["betas"], seed=3, rng="philox")
    ref = oracle.Sim(c["graph"], c["betas"], seed=3, rng="philox")
    dev.run(5, 1)
    ref.run(5, 1)
    st, r = dev.read_state(), ref.read()
    assert np.array_equal(st["spins"], r["spins"]) and np.array_equal(st["energy"], r["energy"])
    dev.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_waits_time_out_and_the_context_survives(ising, kind):
    assert ising.ERRORS[ising.ising_selftest_wait(kind)] == "TIMEOUT"
    _still_works(ising)


def test_allocation_cap_reports_oom_and_lifts(ising):
    c = W.config0()
    ising.ising_set_alloc_cap(4096)
    try:
        with pytest.raises(ising.IsingError) as e:
            ising.Ising(c["graph"], c["betas"], seed=3, rng="philox")
        assert e.value.name == "OOM"
        with pytest.raises(ising.IsingError) as e:
            ising.Mlp(8, seed=1)
        assert e.value.name == "OOM"
    finally:
        ising.ising_set_alloc_cap(0)
    _still_works(ising)


def test_selftest_rejects_unknown_kind(ising):
    assert ising.ERRORS[ising.ising_selftest_wait(7)] == "INVALID_ARG"


def test_measured_latencies_are_plausible(ising):
    lat = ising.ising_measure_latencies()
    assert 5.0 < lat["shared_load"] < 300.0, lat
    assert 1.0 < lat["int_mad"] < 40.0, lat
    assert 5.0 < lat["shuffle"] < 300.0, lat
    assert 2.0 < lat["barrier_8_warps"] < 1000.0, lat
