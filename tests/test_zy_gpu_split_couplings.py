"""Split couplings (ising_set_trotter) against the oracle's split mode (GPU).

Temperature k weights a state by exp(-beta_k E_space - K_k C), C the negated
sum over Trotter pairs; flips look (k_s, k_tau) up in a host-built table and
PT swaps evaluate the deterministic exponential on the device.  Every check is
element by element: spins, spatial fields, spatial energies, Trotter sums,
labels, acceptance counts and counters.

This file is collected after every other GPU file but the allocation-free run's
(which comes last), so that a run stopping at its first failure has already run
the rest.
"""
from __future__ import annotations

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


trotter_K = W.trotter_couplings


def assert_same(dev, ref, what=""):
    d, r = dev.read_state(), ref.read()
    assert np.array_equal(d["spins"], r["spins"]), f"spins {what}"
    assert np.array_equal(d["fields"], r["fields"]), f"fields {what}"
    assert np.array_equal(d["energy"], r["energy"]), f"energy {what}"
    assert np.array_equal(dev.read_trotter(), ref.read_trotter()), f"Trotter sums {what}"
    assert np.array_equal(d["temp_of_slot"], r["temp_of_slot"]), f"labels {what}"
    assert (d["sweeps"], d["passes"]) == (r["sweeps"], r["passes"]), f"counters {what}"
    if dev.R > 1:
        assert np.array_equal(dev.swap_stats(), r["swap_acc"]), f"swap counts {what}"


def split_pair(ising, g, betas, K, seed, rng, field_bits, flags=None):
    dev = ising.Ising(g, betas, seed=seed, rng=rng, field_bits=field_bits)
    if flags is not None:
        dev.set_launch(0, 0, flags)
    dev.set_trotter(K)
    ref = oracle.Sim(g, betas, seed=seed, rng=rng, threads=4)
    ref.set_trotter(K)
    assert_same(dev, ref, "after set_trotter")
    return dev, ref


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
@pytest.mark.parametrize("fb", [16, 32])
def test_split_chain_with_pt_matches_the_oracle(ising, rng, fb):
    """8x8 lattice x 16 slices, 12 temperatures, K from a transverse field:
    persistent launches with the PT pass fused, and per-sweep launches with a
    separate PT kernel, both bit-exact over sweeps and swaps."""
    g = W.layered_graph(8, 16, graph_seed=3)
    betas = W.geometric_betas(12, 0.1, 3.0)
    K = trotter_K(betas, 2.0, 16)
    for flags in (1, 0):
        dev, ref = split_pair(ising, g, betas, K, 5489, rng, fb, flags)
        assert dev.info()["fast_kernel"] == 2
        for n, every in ((10, 1), (6, 2), (3, 0)):
            dev.run(n, every)
            ref.run(n, every)
            assert_same(dev, ref, f"flags {flags} after ({n}, {every})")
        assert dev.swap_stats().sum() > 0
        dev.close()


def test_split_separate_sweep_and_pt_calls(ising):
    g = W.layered_graph(6, 8, graph_seed=9)
    betas = W.geometric_betas(9, 0.2, 2.5)
    K = trotter_K(betas, 1.5, 8)
    dev, ref = split_pair(ising, g, betas, K, 31, "mt19937", 32)
    for k in range(5):
        dev.sweep(k + 1)
        ref.sweep(k + 1)
        dev.pt_swap()
        ref.pt_swap()
    assert_same(dev, ref)


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_config1_first_sweeps(ising, rng):
    """The 32x32 x 32-slice, 256-replica workload under split couplings (the
    bench path: one persistent launch with fused PT), 12 sweeps."""
    c = W.config1_trotter()
    dev, ref = split_pair(ising, c["graph"], c["betas"], c["K"], c["seed"], rng, 16)
    assert dev.info()["persistent_ok"] == 1
    dev.run(12, 1)
    ref.run(12, 1)
    assert_same(dev, ref)


@pytest.mark.parametrize("L,M,fb", [(3, 64, 32), (3, 96, 16)])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_long_columns(ising, L, M, fb, rng):
    """M a multiple of 32 above 32 (the long-column instantiation)."""
    g = W.layered_graph(L, M, graph_seed=L * 100 + M, j_tau=3)
    betas = W.geometric_betas(7, 0.1, 2.0)
    K = trotter_K(betas, 3.0, M)
    dev, ref = split_pair(ising, g, betas, K, 4242 + M, rng, fb)
    dev.run(5, 1)
    ref.run(5, 1)
    assert_same(dev, ref)


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_many_small_replicas(ising, rng):
    """700 replicas of an 8x8 x 16 model: two columns per thread in blocks of
    at most 128 threads (the small-block instantiation)."""
    g = W.layered_graph(8, 16, graph_seed=12)
    betas = W.geometric_betas(700, 0.1, 3.0)
    K = trotter_K(betas, 2.0, 16)
    dev, ref = split_pair(ising, g, betas, K, 99, rng, 16)
    assert dev.info()["threads_per_block"] <= 128
    dev.run(4, 1)
    ref.run(4, 1)
    assert_same(dev, ref)


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_reproduces_the_plain_chain_where_the_rules_coincide(ising, rng):
    """K_k = beta_k j_tau at dyadic temperatures: every exponent is the same
    FP64 number as without split couplings, so the two device chains agree
    bit for bit (spins, labels; E_plain = E_space + j_tau C)."""
    g = W.layered_graph(6, 16, graph_seed=21, j_tau=4)
    betas = np.array([0.125, 0.25, 0.375, 0.5, 0.75, 1.0])
    plain = ising.Ising(g, betas, seed=77, rng=rng, field_bits=32)
    split = ising.Ising(g, betas, seed=77, rng=rng, field_bits=32)
    split.set_trotter(4.0 * betas)
    plain.run(30, 1)
    split.run(30, 1)
    a, b = plain.read_state(), split.read_state()
    assert np.array_equal(a["spins"], b["spins"])
    assert np.array_equal(a["temp_of_slot"], b["temp_of_slot"])
    assert np.array_equal(a["energy"], b["energy"] + 4 * split.read_trotter())
    assert np.array_equal(plain.swap_stats(), split.swap_stats())


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_checkpoint_resume_is_bit_exact(ising, rng):
    """Save after 7 sweeps, load into a fresh handle without split couplings
    (the blob sets them), run 5 more on both: identical to each other and to
    the oracle; a plain blob is refused by a handle with split couplings."""
    g = W.layered_graph(6, 8, graph_seed=40)
    betas = W.geometric_betas(10, 0.1, 2.5)
    K = trotter_K(betas, 2.0, 8)
    dev, ref = split_pair(ising, g, betas, K, 17, rng, 16)
    dev.run(7, 1)
    ref.run(7, 1)
    blob = dev.save()
    other = ising.Ising(g, betas, seed=999, rng=rng, field_bits=16)
    other.load(blob)
    for h in (dev, other):
        h.run(5, 1)
    ref.run(5, 1)
    assert_same(dev, ref, "resumed run")
    assert_same(other, ref, "loaded handle")
    plain = ising.Ising(g, betas, seed=17, rng=rng, field_bits=16)
    with pytest.raises(ising.IsingError) as e:
        dev.load(plain.save())
    assert e.value.name == "INVALID_ARG"
    for h in (dev, other, plain):
        h.close()


def test_philox_checkpoint_carries_the_generator_key(ising):
    """Philox words depend on (seed, instance): a blob loaded into a handle
    initialised with another seed continues the saved chain (plain couplings)."""
    c = W.config0()
    a = ising.Ising(c["graph"], c["betas"], seed=11, rng="philox", field_bits=16)
    a.run(9, 1)
    b = ising.Ising(c["graph"], c["betas"], seed=999, rng="philox", field_bits=16)
    b.load(a.save())
    a.run(6, 1)
    b.run(6, 1)
    ref = oracle.Sim(c["graph"], c["betas"], seed=11, rng="philox", threads=4)
    ref.run(15, 1)
    for h in (a, b):
        d, r = h.read_state(), ref.read()
        for key in ("spins", "fields", "energy", "temp_of_slot"):
            assert np.array_equal(d[key], r[key]), key
        h.close()


def test_split_refusals(ising):
    """Models without the lean kernel, a second call and the allocation-free
    run are refused; without split couplings C reads 0."""
    g = W.random_graph(12, 20, seed=1)
    dev = ising.Ising(g, [0.3, 0.6], seed=1)
    with pytest.raises(ising.IsingError) as e:
        dev.set_trotter([0.5, 0.4])
    assert e.value.name == "UNSUPPORTED"
    assert np.array_equal(dev.read_trotter(), [0, 0])
    dev.run(3, 1)  # still usable with plain couplings
    dev.close()
    c = W.config0()
    dev = ising.Ising(c["graph"], c["betas"], seed=2, rng="philox")
    dev.set_trotter(trotter_K(c["betas"], 2.0, 16))
    with pytest.raises(ising.IsingError) as e:
        dev.set_trotter(trotter_K(c["betas"], 2.0, 16))
    assert e.value.name == "INVALID_ARG"
    with pytest.raises(ising.IsingError) as e:
        ising.ising_run_noalloc(dev.h, 2, 1)
    assert e.value.name == "UNSUPPORTED"
    dev.close()
