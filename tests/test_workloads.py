"""The seeded synthetic inputs have the shapes and value ranges of the
workloads they stand in for (section 4 of the paper; the paper's QMC models
themselves are not available): layered lattices with two partial matchings,
integer couplings and fields, the Trotter ring, geometric ladders, and the
ragged batch's size distribution.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1004_0024_gb300 import workloads as W


def _edges(g):
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return rows, g.col, g.J


def _check_layered(g, L, Ly, M, j_tau=4):
    S = L * Ly
    assert g.n == S * M and g.n_slices == M and g.slice_size == S
    rows, cols, J = _edges(g)
    same_slice = rows // S == cols // S
    # spatial part: degree 4 (lattice) plus at most 2 matching partners
    sp_deg = np.bincount(rows[same_slice], minlength=g.n)
    assert sp_deg.min() >= 4 and sp_deg.max() <= 6
    assert set(np.unique(J[same_slice]).tolist()) <= {-3, -2, -1, 1, 2, 3}
    # the Trotter ring: same site, adjacent slices, coupling j_tau
    tau = ~same_slice
    assert np.all(cols[tau] % S == rows[tau] % S)
    dt = (cols[tau] // S - rows[tau] // S) % M
    assert set(np.unique(dt).tolist()) <= {1, M - 1}
    assert np.all(J[tau] == j_tau)
    if M >= 3:
        assert np.all(np.bincount(rows[tau], minlength=g.n) == 2)
    assert set(np.unique(g.h).tolist()) <= {-2, -1, 0, 1, 2}
    # every slice carries the same spatial model
    for t in range(1, M):
        assert np.array_equal(g.h[t * S:(t + 1) * S], g.h[:S])
    # symmetric couplings
    pairs = dict(zip(zip(rows.tolist(), cols.tolist()), J.tolist()))
    assert all(pairs[(j, i)] == v for (i, j), v in pairs.items())
    return sp_deg[:S] - 4  # matching partners per site


@pytest.mark.parametrize("cfg,L,Ly,M,R,lo,hi", [
    (W.config0, 8, 8, 16, 32, 0.1, 3.0),
    (W.config1, 32, 32, 32, 256, 0.05, 5.0),
])
def test_named_configs_have_their_shapes(cfg, L, Ly, M, R, lo, hi):
    c = cfg()
    extra = _check_layered(c["graph"], L, Ly, M)
    # two partial matchings, each covering about half of the sites
    assert 0.6 < extra.mean() < 1.4
    b = np.asarray(c["betas"])
    assert b.size == R == c["R"] and b[0] == pytest.approx(lo) and b[-1] == pytest.approx(hi)
    assert np.allclose(b[1:] / b[:-1], (hi / lo) ** (1.0 / (R - 1)))


def test_many_replica_and_paper_shaped_configs():
    c3 = W.config3()
    _check_layered(c3["graph"], 16, 16, 16)
    assert c3["R"] == 65536 and len(c3["betas"]) == 65536
    cp = W.config_paper()
    _check_layered(cp["graph"], 8, 12, 256)
    assert cp["graph"].n == 24576 and cp["R"] == 115 and cp["sweeps"] == 30000


def test_ragged_batch_distribution():
    d = W.ragged_instances(4096)
    assert len(d) == 4096 and [x["index"] for x in d] == list(range(4096))
    M = np.array([x["M"] for x in d])
    L = np.array([x["L"] for x in d])
    R = np.array([x["R"] for x in d])
    N = L * L * M
    assert set(np.unique(M).tolist()) == {16, 32}
    assert L.min() >= 8 and L.max() <= 32
    assert R.min() >= 8 and R.max() <= 64
    # spin counts log-uniform over 2^11 .. 2^15 (up to the clamp and rounding of L)
    lg = np.log2(N)
    assert lg.min() >= 10.0 and lg.max() <= 15.1
    assert 12.3 < lg.mean() < 13.4
    # reproducible: the same seed gives the same batch
    assert W.ragged_instances(4096) == d


def test_split_coupling_workload():
    """cfg1 with K_k = (1/2) ln coth(beta_k Gamma / M), Gamma = 2, M = 32:
    positive, falling as beta rises, from 2.88 at beta 0.05 to 0.60 at 5.0."""
    c = W.config1_trotter()
    K = c["K"]
    assert K.shape == (256,) and np.all(np.diff(K) < 0) and np.all(K > 0)
    assert K[0] == pytest.approx(2.8842, abs=1e-3) and K[-1] == pytest.approx(0.5975, abs=1e-3)
    # the mapping's defining identity: tanh(K) = exp(-2 beta Gamma / M)
    assert np.allclose(np.tanh(K), np.exp(-2.0 * c["betas"] * 2.0 / 32))


@pytest.mark.parametrize("L,Ly,seed", [(8, 8, 1), (32, 32, 1), (8, 12, 7), (16, 16, 3)])
def test_matchings_are_disjoint_and_off_the_lattice(L, Ly, seed):
    """The spatial edges beyond the periodic lattice come from two partial
    matchings (section 1: degree 6-8 with the Trotter pair): none of them is a
    lattice bond or a self loop, no site has more than two such partners (one
    per matching), and each matching stops at a quarter of the sites in pairs."""
    adj, Jd, h = W.spatial_model(L, seed, Ly)
    S = L * Ly

    def site(x, y):
        return (y % Ly) * L + (x % L)

    lattice = set()
    for y in range(Ly):
        for x in range(L):
            a = site(x, y)
            for b in (site(x + 1, y), site(x, y + 1)):
                lattice.add((min(a, b), max(a, b)))
    assert len(lattice) == 2 * S
    edges = {(min(a, b), max(a, b)) for a in range(S) for b in adj[a]}
    assert lattice <= edges and set(Jd) == edges
    extra = edges - lattice
    partners = np.zeros(S, dtype=np.int64)
    for a, b in extra:
        assert a != b
        partners[a] += 1
        partners[b] += 1
    assert partners.max() <= 2
    # each matching accepts floor(S / 4) pairs (about half of the sites covered)
    assert len(extra) == 2 * (S // 4)
    assert h.shape == (S,)
