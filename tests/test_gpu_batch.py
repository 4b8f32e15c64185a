"""Ragged batches: every instance bit-exact against its own oracle run (GPU).

Instance b of a batch must equal an oracle simulation of its model, ladder and
seed with Philox instance id b.
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


def _mixed_instances():
    """Layered models of several slice counts and sizes, an unstructured graph,
    a 64-slice model (the lean kernel's long columns) and a 33-slice model
    (generic kernel), with ragged replica counts."""
    specs = [(8, 16, 8), (8, 32, 13), (9, 16, 32), (10, 16, 20), (12, 8, 5), (16, 16, 9),
             (3, 4, 3), (4, 5, 7), (3, 64, 4), (11, 32, 24), (8, 16, 1), (6, 16, 40), (3, 33, 5)]
    out = []
    for k, (L, M, R) in enumerate(specs):
        g = W.layered_graph(L, M, graph_seed=700 + k)
        out.append((g, W.geometric_betas(R, 0.1, 3.0), 9000 + 17 * k))
    out.append((W.random_graph(40, 90, seed=5), W.geometric_betas(6, 0.2, 1.5), 4321))
    return out


def _check_instance(batch, k, inst, rng, schedule):
    g, betas, seed = inst
    ref = oracle.Sim(g, betas, seed=seed, rng=rng, instance=k)
    for n, every in schedule:
        ref.run(n, every)
    d, r = batch.read_state(k), ref.read()
    for key in ("spins", "fields", "energy", "temp_of_slot"):
        assert np.array_equal(d[key], r[key]), (k, key, batch.info(k))
    assert (d["sweeps"], d["passes"]) == (r["sweeps"], r["passes"]), k
    if len(betas) > 1:
        assert np.array_equal(batch.swap_stats(k), r["swap_acc"]), k


@pytest.mark.parametrize("rng", ["philox", "mt19937"])
def test_mixed_batch_bit_exact(ising, rng):
    inst = _mixed_instances()
    b = ising.Batch(inst, rng=rng, field_bits=16)
    kinds = {(b.info(k)["resident"], b.info(k)["fast_kernel"]) for k in range(len(inst))}
    assert (1, 1) in kinds and (0, 2) in kinds and (0, 0) in kinds  # resident, lean, generic
    schedule = [(7, 1), (5, 2), (3, 0)]
    for n, every in schedule:
        b.run(n, every)
    b.run(7, 1)  # replay of a recorded graph
    for k in range(len(inst)):
        _check_instance(b, k, inst[k], rng, schedule + [(7, 1)])
    b.close()


def _packed_instances():
    """Layered models the packed kernel takes (M in {8, 16, 32}), several
    lattices and ragged ladders: a batch of them runs as persistent waves."""
    specs = [(8, 16, 8), (8, 32, 13), (9, 16, 32), (10, 16, 20), (12, 8, 5), (16, 16, 9), (6, 8, 3),
             (11, 32, 24), (8, 16, 1), (6, 16, 40), (14, 32, 7)]
    return [(W.layered_graph(L, M, graph_seed=800 + k), W.geometric_betas(R, 0.1, 3.0), 7000 + 13 * k)
            for k, (L, M, R) in enumerate(specs)]


@pytest.mark.parametrize("rng", ["philox", "mt19937"])
@pytest.mark.parametrize("per_sweep", [False, True])
def test_packed_batch_bit_exact(ising, rng, per_sweep):
    """Persistent waves (one cooperative launch per wave and call, PT fused per
    instance) and the per-sweep launches of the same batch: every instance
    bit-exact against its oracle run, over calls with PT after every sweep,
    every second sweep (with a remainder) and none."""
    inst = _packed_instances()
    b = ising.Batch(inst, rng=rng, field_bits=16, per_sweep=per_sweep)
    kinds = {(b.info(k)["resident"], b.info(k)["fast_kernel"]) for k in range(len(inst))}
    if not per_sweep:
        assert kinds == {(1, 4)}, kinds
    else:
        assert all(kind != 4 for _, kind in kinds), kinds
    schedule = [(7, 1), (5, 2), (3, 0), (7, 1)]
    for n, every in schedule:
        b.run(n, every)
    for k in range(len(inst)):
        _check_instance(b, k, inst[k], rng, schedule)
    b.close()


def test_autotune_changes_speed_not_results(ising):
    inst = _mixed_instances()[:8]
    b = ising.Batch(inst, rng="philox", field_bits=16)
    b.run(4, 1)
    b.autotune()
    b.run(9, 1)
    for k in range(len(inst)):
        _check_instance(b, k, inst[k], "philox", [(4, 1), (9, 1)])
    b.close()


def test_full_ragged_workload_sampled_parity(ising):
    """4096 instances (spin counts log-uniform in 2^11..2^15, 8..64 replicas),
    100 sweeps + PT per instance, in persistent waves; bit-exact on 64
    sampled instances plus the smallest and the largest, fields/energies
    consistent elsewhere."""
    descs = W.ragged_instances(4096)
    built = [W.build_instance(d) for d in descs]
    inst = [(x["graph"], x["betas"], x["seed"]) for x in built]
    b = ising.Batch(inst, rng="philox", field_bits=16)
    b.autotune()
    b.run(100, 1)
    assert all(b.info(k)["fast_kernel"] == 4 for k in range(0, len(inst), 97))  # persistent waves
    sizes = [x["graph"].n for x in built]
    rng = np.random.default_rng(11)
    sample = set(rng.choice(len(inst), 64, replace=False).tolist())
    sample |= {int(np.argmin(sizes)), int(np.argmax(sizes))}
    for k in sorted(sample):
        _check_instance(b, k, inst[k], "philox", [(100, 1)])
    for k in rng.choice(len(inst), 16, replace=False).tolist():
        g = inst[k][0]
        st = b.read_state(k)
        r = int(rng.integers(0, st["spins"].shape[0]))
        assert np.array_equal(oracle.fields(g, st["spins"][r]), st["fields"][r])
        assert oracle.energy(g, st["spins"][r]) == st["energy"][r]
    b.close()
