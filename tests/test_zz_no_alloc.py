"""ising_run_noalloc: the allocation-free run, for callers that cannot allocate
device memory while they run, must reproduce ising_run exactly (GPU).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_1004_0024_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ising():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1004_0024_gb300 import ising as mod
    return mod


def _same(a, b):
    sa, sb = a.read_state(), b.read_state()
    for key in ("spins", "fields", "energy", "temp_of_slot", "sweeps", "passes"):
        assert np.array_equal(np.asarray(sa[key]), np.asarray(sb[key])), key
    assert np.array_equal(a.swap_stats(), b.swap_stats())


def test_noalloc_run_matches_run_on_two_calls_in_a_row(ising):
    c = W.config0()
    ref = ising.Ising(c["graph"], c["betas"], seed=97, rng="philox", field_bits=16)
    dut = ising.Ising(c["graph"], c["betas"], seed=97, rng="philox", field_bits=16)
    assert dut.info()["persistent_ok"] == 1
    for n, every in ((9, 1), (13, 2)):  # 13 = 6 fused groups + 1 trailing sweep
        ref.run(n, every)
        ising.ising_run_noalloc(dut.h, n, every)
        _same(ref, dut)


def test_noalloc_run_on_the_large_model(ising):
    c = W.config1()
    ref = ising.Ising(c["graph"], c["betas"], seed=5, rng="philox", field_bits=16)
    dut = ising.Ising(c["graph"], c["betas"], seed=5, rng="philox", field_bits=16)
    for _ in range(2):
        ref.run(6, 1)
        ising.ising_run_noalloc(dut.h, 6, 1)
        _same(ref, dut)


def test_noalloc_run_at_the_largest_replica_count(ising):
    # The static energy exchange holds 2 x 16384 energies.  Every block of the
    # persistent launch also keeps the whole ladder's labels in shared memory,
    # so the largest ladder that can run persistently is smaller than that on
    # any model: R = 16384 must then be refused as UNSUPPORTED (no persistent
    # launch), and the largest ladder that is persistent (a small model, a PT
    # pass after every sweep) must match ising_run.
    g = W.graph_from_edges(4, {(0, 1): 1, (1, 2): -1, (2, 3): 2, (0, 3): -2}, [1, 0, -1, 0])
    top = ising.Ising(g, W.geometric_betas(16384, 0.1, 2.0), seed=3, rng="philox", field_bits=16)
    if top.info()["persistent_ok"] == 0:
        with pytest.raises(ising.IsingError) as ei:
            ising.ising_run_noalloc(top.h, 2, 1)
        assert ei.value.name == "UNSUPPORTED"
    top.close()
    R = next(r for r in (16384, 8192, 6144, 4096, 3072, 2048, 1024)
             if ising.Ising(g, W.geometric_betas(r, 0.1, 2.0), seed=3, rng="philox",
                            field_bits=16).info()["persistent_ok"] == 1)
    betas = W.geometric_betas(R, 0.1, 2.0)
    ref = ising.Ising(g, betas, seed=3, rng="philox", field_bits=16)
    dut = ising.Ising(g, betas, seed=3, rng="philox", field_bits=16)
    for _ in range(2):
        ref.run(4, 1)
        ising.ising_run_noalloc(dut.h, 4, 1)
        _same(ref, dut)
    assert dut.stats()["sweep_launches"] == 2


def test_noalloc_rejects_what_it_cannot_serve(ising):
    g = W.graph_from_edges(4, {(0, 1): 1, (1, 2): -1, (2, 3): 2}, [1, 0, -1, 0])
    big = ising.Ising(g, W.geometric_betas(16385, 0.1, 2.0), seed=1, rng="philox", field_bits=16)
    with pytest.raises(ising.IsingError) as ei:
        ising.ising_run_noalloc(big.h, 1, 1)
    assert ei.value.name == "INVALID_ARG"
    big.close()
    mt = ising.Ising(g, W.geometric_betas(8, 0.1, 2.0), seed=1, rng="mt19937", field_bits=16)
    with pytest.raises(ising.IsingError) as ei:
        ising.ising_run_noalloc(mt.h, 1, 1)
    assert ei.value.name == "UNSUPPORTED"
