"""Bit-exact parity of the CUDA path with the oracle (GPU).

Every comparison is element by element on spins, local fields, energies,
temperature labels, PT acceptance counts and sweep/pass counters.  Inputs come
from ``paper_1004_0024_gb300.workloads`` (seeded, synthetic).
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


def assert_same(dev, ref, what=""):
    d, r = dev.read_state(), ref.read()
    assert np.array_equal(d["spins"], r["spins"]), f"spins {what}"
    assert np.array_equal(d["fields"], r["fields"]), f"fields {what}"
    assert np.array_equal(d["energy"], r["energy"]), f"energy {what}"
    assert np.array_equal(d["temp_of_slot"], r["temp_of_slot"]), f"labels {what}"
    assert (d["sweeps"], d["passes"]) == (r["sweeps"], r["passes"]), f"counters {what}"
    if dev.R > 1:
        assert np.array_equal(dev.swap_stats(), r["swap_acc"]), f"swap counts {what}"


def pair(ising, g, betas, seed, rng, field_bits, launch=None):
    dev = ising.Ising(g, betas, seed=seed, rng=rng, field_bits=field_bits)
    if launch is not None:
        dev.set_launch(*launch)
    ref = oracle.Sim(g, betas, seed=seed, rng=rng)
    assert_same(dev, ref, "after init")
    return dev, ref


# ------------------------------------------------------------ named configs
def test_config0_1000_sweeps_pt_every_sweep_mt19937(ising):
    c = W.config0()
    dev, ref = pair(ising, c["graph"], c["betas"], c["seed"], "mt19937", 32)
    for chunk in range(4):
        dev.run(250, 1)
        ref.run(250, 1)
        assert_same(dev, ref, f"after {250 * (chunk + 1)} sweeps")


def test_config0_philox(ising):
    c = W.config0()
    dev, ref = pair(ising, c["graph"], c["betas"], c["seed"], "philox", 32)
    dev.run(300, 1)
    ref.run(300, 1)
    assert_same(dev, ref)


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_config1_first_20_sweeps(ising, rng):
    c = W.config1()
    dev, ref = pair(ising, c["graph"], c["betas"], c["seed"], rng, 16)
    for _ in range(4):
        dev.run(5, 1)
        ref.run(5, 1)
        assert_same(dev, ref)


def test_config1_full_200_sweeps_bit_exact(ising):
    """The full 32768-spin x 256-replica run (200 sweeps + PT), as timed by bench.py."""
    c = W.config1()
    dev, ref = pair(ising, c["graph"], c["betas"], c["seed"], "mt19937", 16)
    dev.run(200, 1)
    ref.run(200, 1)
    assert_same(dev, ref)
    st = dev.read_state()
    g = c["graph"]
    for r in (0, 77, 255):  # fields and energy recomputed from scratch
        assert np.array_equal(oracle.fields(g, st["spins"][r]), st["fields"][r])
        assert oracle.energy(g, st["spins"][r]) == st["energy"][r]


# --------------------------------------------------------- shapes and edges
@pytest.mark.parametrize("n,edges,R", [(1, 0, 1), (2, 1, 2), (3, 3, 3), (5, 7, 7), (17, 40, 4),
                                       (100, 300, 5), (1000, 2500, 6)])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_unstructured_graphs(ising, n, edges, R, rng):
    g = W.random_graph(n, edges, seed=n + edges)
    betas = W.geometric_betas(R, 0.2, 1.5)
    dev, ref = pair(ising, g, betas, 99 + n, rng, 32 if n % 2 else 16)
    dev.run(7, 2)
    ref.run(7, 2)
    assert_same(dev, ref)


@pytest.mark.parametrize("L,M", [(3, 2), (3, 3), (4, 4), (3, 5), (5, 8), (4, 33), (3, 64)])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_slice_counts(ising, L, M, rng):
    g = W.layered_graph(L, M, graph_seed=L * 100 + M, j_tau=3)
    betas = W.geometric_betas(9, 0.1, 2.0)
    dev, ref = pair(ising, g, betas, 4242, rng, 16)
    dev.run(9, 1)
    ref.run(9, 1)
    assert_same(dev, ref)


@pytest.mark.parametrize("G,T", [(1, 32), (2, 64), (4, 128), (8, 256), (1, 1024), (8, 64),
                                 (2, 32)])
@pytest.mark.parametrize("flags", [0, 1, 2, 4, 5])
def test_launch_shapes_give_identical_results(ising, G, T, flags):
    """Every accepted launch shape and kernel path gives the same chain (flags:
    1 persistent launch with fused PT, 2 generic kernel, 4 no lean variant;
    0 and 4 are per-sweep launches)."""
    c = W.config0()
    betas = W.geometric_betas(30, 0.1, 3.0)  # 30 replicas: ragged last block
    for rng in ("mt19937", "philox"):
        dev, ref = pair(ising, c["graph"], betas, 7, rng, 16, launch=(G, T, flags))
        info = dev.info()
        if flags == 2:
            assert info["fast_kernel"] == 0
        dev.run(25, 1)
        ref.run(25, 1)
        assert_same(dev, ref, f"{rng} {info}")
        dev.run(7, 3)
        ref.run(7, 3)
        assert_same(dev, ref, f"{rng} {info}")


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_config1_paths_agree(ising, rng):
    """cfg1 through every kernel (track, packed, lean, register-resident,
    generic), persistent with fused PT (the bench path) or per-sweep
    launches: identical to the oracle after 12 sweeps."""
    c = W.config1()
    ref = oracle.Sim(c["graph"], c["betas"], seed=c["seed"], rng=rng)
    ref.run(12, 1)
    for flags, kernel in ((9, 3), (8, 3), (1, 4), (0, 4), (17, 2), (16, 2), (5, 1), (4, 1), (2, 0)):
        dev = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng=rng, field_bits=16)
        dev.set_launch(0, 0, flags)
        info = dev.info()
        assert info["fast_kernel"] == kernel
        assert info["persistent_ok"] == (flags & 1)
        dev.run(12, 1)
        assert_same(dev, ref, f"flags {flags}")
        dev.close()


def test_separate_sweep_and_pt_calls(ising):
    c = W.config0()
    dev, ref = pair(ising, c["graph"], c["betas"][:13], 31, "mt19937", 32)
    for k in range(6):
        dev.sweep(k + 1)
        ref.sweep(k + 1)
        dev.pt_swap()
        ref.pt_swap()
        dev.pt_swap()
        ref.pt_swap()
    assert_same(dev, ref)
    dev.run(10, 3)
    ref.run(10, 3)
    assert_same(dev, ref)


def test_zero_model_and_isolated_spins(ising):
    g = W.graph_from_edges(64, {}, np.zeros(64))
    dev, ref = pair(ising, g, [0.5, 1.0, 2.0], 3, "mt19937", 32)
    s0 = dev.read_state()["spins"]
    dev.sweep(1)
    assert np.array_equal(dev.read_state()["spins"], -s0)
    h = np.arange(-4, 4)
    g2 = W.graph_from_edges(8, {}, h)
    dev, ref = pair(ising, g2, [0.3, 0.9], 5, "philox", 16)
    dev.run(5, 1)
    ref.run(5, 1)
    assert_same(dev, ref)
    assert np.array_equal(dev.read_state()["fields"][0], h)


def test_checkpoint_resume_is_bit_exact(ising):
    c = W.config0()
    a = ising.Ising(c["graph"], c["betas"], seed=11, rng="mt19937", field_bits=16)
    a.run(10, 1)
    blob = a.save()
    b = ising.Ising(c["graph"], c["betas"], seed=999, rng="mt19937", field_bits=16)
    b.load(blob)
    a.run(10, 1)
    b.run(10, 1)
    sa, sb = a.read_state(), b.read_state()
    for k in ("spins", "fields", "energy", "temp_of_slot"):
        assert np.array_equal(sa[k], sb[k])
    ref = oracle.Sim(c["graph"], c["betas"], seed=11)
    ref.run(20, 1)
    assert_same(b, ref)


def test_set_seed_continues_with_the_new_seeds_random_numbers(ising):
    # a fresh handle of seed 11 given seed 23: its chain is the oracle's chain
    # of seed 23 started from the seed-11 handle's initial spins
    c = W.config0()
    dev = ising.Ising(c["graph"], c["betas"], seed=11, rng="philox", field_bits=32)
    init = dev.read_state()["spins"]
    dev.set_seed(23)
    ref = oracle.Sim(c["graph"], c["betas"], seed=23, rng="philox")
    ref.set_spins(init)
    assert_same(dev, ref, "after set_seed")
    dev.run(40, 1)
    ref.run(40, 1)
    assert_same(dev, ref, "40 sweeps after set_seed")
    # after loading a checkpoint, the reseeded chain leaves the saved chain's path
    blob = dev.save()
    a = ising.Ising(c["graph"], c["betas"], seed=5, rng="philox", field_bits=32)
    b = ising.Ising(c["graph"], c["betas"], seed=5, rng="philox", field_bits=32)
    a.load(blob)
    b.load(blob)
    b.set_seed(77)
    a.run(5, 1)
    b.run(5, 1)
    dev.run(5, 1)
    assert np.array_equal(a.read_state()["spins"], dev.read_state()["spins"])
    assert not np.array_equal(b.read_state()["spins"], dev.read_state()["spins"])
    mt = ising.Ising(c["graph"], c["betas"], seed=5, rng="mt19937", field_bits=32)
    with pytest.raises(ising.IsingError) as ei:
        mt.set_seed(3)
    assert ei.value.name == "UNSUPPORTED"


def test_graph_replay_matches_fresh_launches(ising):
    """ising_run records a CUDA graph once and replays it; replays must advance
    the device-side counters and streams exactly like fresh launches."""
    c = W.config0()
    dev, ref = pair(ising, c["graph"], c["betas"], 17, "philox", 16)
    for _ in range(5):
        dev.run(4, 2)
        ref.run(4, 2)
    assert_same(dev, ref)


def test_not_initialised_is_reported(ising):
    g = W.layered_graph(3, 3, 1)
    h = ising.ising_create(g.n, g.row_ptr, g.col, g.J, g.h, 3)
    with pytest.raises(ising.IsingError) as ei:
        ising.ising_run(h, 5, 1)
    assert ei.value.name == "NOT_INITIALISED"
    ising.ising_destroy(h)


@pytest.mark.parametrize("rng", ["philox", "mt19937"])
def test_config3_sampled_replicas(ising, rng):
    """The 4096-spin x 65536-replica throughput workload: without PT every
    replica is an independent chain, so the first 16 slots are checked
    against an oracle run of those 16 replicas alone; the swap tables of this
    ladder exceed 2^28 entries, so PT is refused and sweeps go on."""
    c = W.config3()
    dev = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng=rng, field_bits=16)
    dev.run(12, 0)
    with pytest.raises(ising.IsingError) as e:
        dev.pt_swap()
    assert e.value.name == "UNSUPPORTED"
    dev.run(8, 0)
    st = dev.read_state()
    ref = oracle.Sim(c["graph"], c["betas"][:16], seed=c["seed"], rng=rng)
    ref.run(20, 0)
    r = ref.read()
    for key in ("spins", "fields", "energy"):
        assert np.array_equal(st[key][:16], r[key]), key
    assert int(st["sweeps"]) == 20
    assert np.array_equal(st["temp_of_slot"], np.arange(c["R"]))
    dev.close()



@pytest.mark.parametrize("L,M,R,rng,fb", [(8, 16, 32, "mt19937", 32), (6, 8, 9, "philox", 16), (5, 4, 6, "mt19937", 16),
                                          (7, 32, 5, "philox", 32), (3, 4, 2, "philox", 16)])
def test_track_kernel_matches_lean_and_oracle(ising, L, M, R, rng, fb):
    """The track-scheduled kernel (opt-in) against the oracle on several slice
    counts, replica counts and field widths, persistent (fused PT) and per
    sweep."""
    g = W.layered_graph(L, M, L + M)
    betas = W.geometric_betas(R, 0.2, 2.5)
    for flags in (9, 8):
        ref = oracle.Sim(g, betas, seed=77, rng=rng)
        dev = ising.Ising(g, betas, seed=77, rng=rng, field_bits=fb)
        dev.set_launch(0, 0, flags)
        assert dev.info()["fast_kernel"] == 3
        for n, every in ((9, 2), (5, 1), (4, 0)):
            dev.run(n, every)
            ref.run(n, every)
            assert_same(dev, ref, f"flags {flags} after ({n}, {every})")
        dev.close()


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
@pytest.mark.parametrize("flags", [-1, 16, 2])
def test_paper_shape_sampled_replicas(ising, rng, flags):
    """The paper's workload shape (96-spin layers, 256 Trotter slices: the
    packed kernel's long columns by default, the lean kernel's with flag 16
    (no packed kernel), the generic kernel with flag 2), 115 replicas without
    PT: the first 6 slots against an oracle run of those replicas alone."""
    c = W.config_paper()
    dev = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng=rng, field_bits=16)
    if flags >= 0:
        dev.set_launch(0, 0, flags)
    assert dev.info()["fast_kernel"] == {-1: 4, 16: 2, 2: 0}[flags]
    dev.run(3, 0)
    dev.run(2, 0)
    st = dev.read_state()
    ref = oracle.Sim(c["graph"], c["betas"][:6], seed=c["seed"], rng=rng)
    ref.run(5, 0)
    r = ref.read()
    for key in ("spins", "fields", "energy"):
        assert np.array_equal(st[key][:6], r[key]), key
    dev.close()


@pytest.mark.parametrize("L,M,fb", [(3, 64, 32), (3, 96, 16), (3, 128, 16), (4, 160, 32), (3, 64, 16),
                                    (5, 256, 16)])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
@pytest.mark.parametrize("path", ["packed", "lean"])
def test_long_columns(ising, L, M, fb, rng, path):
    """M a multiple of 32 above 32: the packed kernel (by default) and the
    lean kernel (flag 16) keep the column as M/32 words and walk them in
    registers (ring wrap at both ends, Trotter bits across word edges); with
    PT after every sweep, bit-exact against the oracle."""
    g = W.layered_graph(L, M, graph_seed=L * 100 + M, j_tau=3)
    betas = W.geometric_betas(9, 0.1, 2.0)
    dev, ref = pair(ising, g, betas, 4242 + M, rng, fb, None if path == "packed" else (0, 0, 16))
    assert dev.info()["fast_kernel"] == (4 if path == "packed" else 2)
    dev.run(7, 1)
    ref.run(7, 1)
    assert_same(dev, ref)
    dev.run(5, 2)
    ref.run(5, 2)
    assert_same(dev, ref, "after 5 more sweeps, PT every second")


@pytest.mark.parametrize("accept", ["fast", "accurate"])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_approximate_exp_acceptance_modes(ising, accept, rng):
    """Flip thresholds built with the paper's fast or accurate exponential
    (section 2.4): sweeps and PT passes bit-exact against the oracle in the
    same mode, and different from the exact mode's chain."""
    g = W.layered_graph(5, 8, graph_seed=31, j_tau=3)
    betas = W.geometric_betas(12, 0.1, 3.0)
    dev = ising.Ising(g, betas, seed=99, rng=rng, field_bits=16, accept=accept)
    ref = oracle.Sim(g, betas, seed=99, rng=rng, accept=accept)
    dev.run(15, 1)
    ref.run(15, 1)
    assert_same(dev, ref)
    exact = oracle.Sim(g, betas, seed=99, rng=rng)
    exact.run(15, 1)
    assert not np.array_equal(exact.read()["spins"], dev.read_state()["spins"])
    dev.close()


def test_reused_word_buffer_gives_the_same_chain(ising):
    """MT19937 word buffers of 256 MB or more (here 10 sweeps of the 32x32x32
    x 256 model, 335 MB) are kept by ising_destroy for the next handle and are
    not zero-filled: a run on the reused buffer equals the same run on a fresh
    one; ising_release_cached_memory empties the cache."""
    c = W.config1()

    def run_once():
        sim = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng="mt19937", field_bits=16)
        sim.run(10, 1)
        st = sim.read_state()
        sim.close()
        return st

    ising.ising_release_cached_memory()
    first = run_once()   # allocates the buffer, then leaves it in the cache
    second = run_once()  # takes it from the cache
    for key in ("spins", "fields", "energy", "temp_of_slot"):
        assert np.array_equal(first[key], second[key]), key
    ising.ising_release_cached_memory()


@pytest.mark.parametrize("L,M,R,fb", [(8, 16, 32, 32), (6, 8, 9, 16), (5, 32, 5, 16), (12, 16, 40, 32),
                                      (9, 8, 3, 32)])
@pytest.mark.parametrize("T", [0, 32, 64, 128, 256])
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_packed_kernel_matches_oracle(ising, L, M, R, fb, T, rng):
    """The packed (slot-scheduled) kernel on several lattices, slice counts,
    ladders, field widths and block sizes (one, two or four warps; 0 =
    automatic), persistent with PT fused and in per-sweep launches, and with
    groups of sweeps between PT passes: bit-exact against the oracle."""
    g = W.layered_graph(L, M, L * 7 + M)
    betas = W.geometric_betas(R, 0.15, 2.8)
    for flags in (1, 0):
        ref = oracle.Sim(g, betas, seed=31 + L, rng=rng)
        dev = ising.Ising(g, betas, seed=31 + L, rng=rng, field_bits=fb)
        dev.set_launch(0, T, flags)
        info = dev.info()
        assert info["fast_kernel"] == 4, info
        if T:
            assert info["threads_per_block"] == T
        for n, every in ((9, 1), (7, 3), (4, 0), (2, 1)):
            dev.run(n, every)
            ref.run(n, every)
            assert_same(dev, ref, f"T {T} flags {flags} after ({n}, {every})")
        dev.close()


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_packed_and_lean_kernels_agree_on_config1(ising, rng):
    """The bench workload through the packed kernel (one and two warps per
    replica) and the lean kernel: the same chain over 30 sweeps with PT."""
    c = W.config1()
    states = []
    for T, flags in ((32, 1), (64, 1), (0, 17)):
        dev = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng=rng, field_bits=16)
        dev.set_launch(0, T, flags)
        assert dev.info()["fast_kernel"] == (2 if flags & 16 else 4)
        dev.run(30, 1)
        states.append(dev.read_state())
        dev.close()
    for st in states[1:]:
        for key in ("spins", "fields", "energy", "temp_of_slot"):
            assert np.array_equal(st[key], states[0][key]), key
