"""Seeded synthetic workloads: layered (Trotter) Ising graphs and temperature ladders.

This module only builds inputs.  It holds none of the sampler's arithmetic
(no random-number generator of the method, no acceptance rule, no field or
energy update) so that the CUDA library and the oracle can both consume
exactly the same graphs.  Its own randomness comes from numpy's PCG64
(``numpy.random.default_rng``), not from the method's MT19937 or Philox.

Graph shape (the paper's QMC setting, sections 1 and 3.1): ``M`` identical
slices ("layers") of an ``L x L`` spatial model, spin ``i = t*L*L + y*L + x``;
each spin is coupled to the corresponding spin of the two neighbouring slices
(ring ``t +- 1 mod M``), so every spin has exactly two Trotter edges, placed
last in its CSR row as in Figure 6.  Spatially each site has its 4 periodic
lattice neighbours plus up to one partner from each of two seeded random
partial matchings (restricted to non-adjacent, not-yet-coupled pairs, each
covering about half of the sites), giving spatial degree 4..6 and total
degree 6..8 (section 1: "each spin is adjacent to 6, 7, or 8 other spins").
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    """CSR Ising model: row i lists (col, J) for every neighbour of spin i."""

    n: int
    row_ptr: np.ndarray  # int32 [n+1]
    col: np.ndarray      # int32 [nnz]
    J: np.ndarray        # int32 [nnz]
    h: np.ndarray        # int32 [n]
    n_slices: int = 1    # M: declared number of identical Trotter slices
    meta: dict = field(default_factory=dict)

    @property
    def slice_size(self) -> int:
        return self.n // max(self.n_slices, 1)

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _csr(n: int, rows: list[list[tuple[int, int]]], h: np.ndarray, n_slices: int, meta=None):
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    for i, r in enumerate(rows):
        row_ptr[i + 1] = row_ptr[i] + len(r)
    col = np.fromiter((c for r in rows for c, _ in r), dtype=np.int32, count=int(row_ptr[-1]))
    J = np.fromiter((j for r in rows for _, j in r), dtype=np.int32, count=int(row_ptr[-1]))
    return Graph(n, row_ptr, col, J, np.asarray(h, dtype=np.int32), n_slices, meta or {})


def spatial_model(L: int, graph_seed: int, Ly: int | None = None):
    """One slice: periodic L x L (or L x Ly) lattice plus two partial matchings.

    Returns (neighbour sets, J dict keyed by (min, max), h per site).  Draw
    order: matching A, matching B, then J per spatial edge in lexicographic
    (min, max) order from {-3,-2,-1,1,2,3}, then h per site from {-2..2}.
    """
    Ly = L if Ly is None else Ly
    if L < 3 or Ly < 3:
        raise ValueError("the lattice sides must be >= 3 so that the 4 lattice neighbours are distinct")
    rng = np.random.default_rng(graph_seed)
    S = L * Ly

    def site(x, y):
        return (y % Ly) * L + (x % L)

    adj = [set() for _ in range(S)]
    for y in range(Ly):
        for x in range(L):
            a = site(x, y)
            for b in (site(x + 1, y), site(x, y + 1)):
                adj[a].add(b)
                adj[b].add(a)
    for _ in range(2):
        perm = rng.permutation(S)
        accepted = 0
        for m in range(S // 2):
            a, b = int(perm[2 * m]), int(perm[2 * m + 1])
            if b in adj[a]:
                continue
            adj[a].add(b)
            adj[b].add(a)
            accepted += 1
            if accepted == S // 4:
                break
    edges = sorted({(min(a, b), max(a, b)) for a in range(S) for b in adj[a]})
    jvals = np.array([-3, -2, -1, 1, 2, 3], dtype=np.int32)
    Jd = {e: int(jvals[rng.integers(0, 6)]) for e in edges}
    h = rng.integers(-2, 3, size=S).astype(np.int32)
    return adj, Jd, h


def layered_graph(L: int, M: int, graph_seed: int, j_tau: int = 4, Ly: int | None = None) -> Graph:
    """M identical copies of ``spatial_model(L, Ly)`` coupled in a Trotter ring."""
    adj, Jd, hs = spatial_model(L, graph_seed, Ly)
    S = L * (L if Ly is None else Ly)
    n = S * M
    # one slice's row template: per site, spatial entries (ascending target)
    # then the Trotter entries; kind 0 = spatial, 1 = slice t-1, 2 = slice t+1,
    # 3 = the other slice of a 2-slice ring
    trot = [1, 2] if M >= 3 else ([3] if M == 2 else [])
    site, kind, tgt, jv = [], [], [], []
    for q in range(S):
        for p in sorted(adj[q]):
            site.append(q); kind.append(0); tgt.append(p); jv.append(Jd[(min(p, q), max(p, q))])
        for k in trot:
            site.append(q); kind.append(k); tgt.append(q); jv.append(j_tau)
    site = np.asarray(site, dtype=np.int64)
    kind = np.asarray(kind, dtype=np.int64)
    tgt = np.asarray(tgt, dtype=np.int64)
    jv = np.asarray(jv, dtype=np.int32)
    t = np.arange(M, dtype=np.int64)[:, None]
    slice_of = np.where(kind == 0, t, np.where(kind == 1, (t - 1) % M,
                        np.where(kind == 2, (t + 1) % M, 1 - t)))
    col = (slice_of * S + tgt[None, :]).astype(np.int32).ravel()
    J = np.tile(jv, M)
    deg = np.bincount(site, minlength=S).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(np.tile(deg, M))
    h = np.tile(hs, M).astype(np.int32)
    return Graph(n, row_ptr, col, J, h, M, dict(L=L, Ly=L if Ly is None else Ly, M=M, graph_seed=graph_seed,
                                                 j_tau=j_tau))


def random_graph(n: int, n_edges: int, seed: int, jmax: int = 3, hmax: int = 2) -> Graph:
    """Unstructured simple graph (for small exact tests): n_edges distinct pairs."""
    rng = np.random.default_rng(seed)
    pairs = set()
    max_edges = n * (n - 1) // 2
    n_edges = min(n_edges, max_edges)
    while len(pairs) < n_edges:
        a, b = rng.integers(0, n, size=2)
        if a != b:
            pairs.add((int(min(a, b)), int(max(a, b))))
    rows: list[list[tuple[int, int]]] = [[] for _ in range(n)]
    for (a, b) in sorted(pairs):
        j = int(rng.integers(1, jmax + 1)) * (1 if rng.integers(0, 2) else -1)
        rows[a].append((b, j))
        rows[b].append((a, j))
    for r in rows:
        r.sort()
    h = rng.integers(-hmax, hmax + 1, size=n).astype(np.int32)
    return _csr(n, rows, h, 1, dict(kind="random", seed=seed))


def graph_from_edges(n: int, edges: dict, h, n_slices: int = 1) -> Graph:
    """CSR from {(a, b): J} with a != b (each pair once)."""
    rows: list[list[tuple[int, int]]] = [[] for _ in range(n)]
    for (a, b), j in edges.items():
        rows[a].append((b, int(j)))
        rows[b].append((a, int(j)))
    for r in rows:
        r.sort()
    return _csr(n, rows, np.asarray(h, dtype=np.int32), n_slices)


def geometric_betas(R: int, lo: float, hi: float) -> np.ndarray:
    """Ascending geometric ladder beta_k = lo * (hi/lo)^(k/(R-1))."""
    if R == 1:
        return np.array([lo], dtype=np.float64)
    return lo * (hi / lo) ** (np.arange(R, dtype=np.float64) / (R - 1))


# ----------------------------------------------------------- named workloads
def config0():
    """8x8 lattice x M=16 (1024 spins), 32 replicas, betas 0.1..3.0, int32 fields."""
    return dict(name="cfg0_L8_M16_R32", graph=layered_graph(8, 16, 1), R=32,
                betas=geometric_betas(32, 0.1, 3.0), seed=5489, field_bits=32, sweeps=1000,
                swap_every=1)


def config1():
    """32x32 lattice x M=32 (32768 spins), 256 replicas, betas 0.05..5.0, int16 fields."""
    return dict(name="cfg1_L32_M32_R256", graph=layered_graph(32, 32, 1), R=256,
                betas=geometric_betas(256, 0.05, 5.0), seed=5489, field_bits=16, sweeps=200,
                swap_every=1)


def trotter_couplings(betas, gamma: float, M: int) -> np.ndarray:
    """K_k = (1/2) ln coth(beta_k Gamma / M): the inter-slice coupling of M
    Trotter slices of a transverse field Gamma at inverse temperature beta_k
    (the standard Suzuki-Trotter mapping; it falls as beta rises)."""
    b = np.asarray(betas, dtype=np.float64)
    return 0.5 * np.log(1.0 / np.tanh(b * gamma / M))


def config1_trotter(gamma: float = 2.0):
    """The 32x32 x 32-slice, 256-replica system with split couplings:
    temperature k weights exp(-beta_k E_space - K_k C), K_k from a transverse
    field Gamma = 2 over the 32 slices (K from 2.88 at beta 0.05 to 0.60 at
    beta 5.0)."""
    c = config1()
    return dict(c, name="cfg1_trotter_L32_M32_R256", K=trotter_couplings(c["betas"], gamma, 32),
                gamma=gamma)


def config3(R: int = 65536):
    """16x16 lattice x M=16 (4096 spins), 65536 replicas, betas 0.1..3.0, int16 fields."""
    return dict(name=f"cfg3_L16_M16_R{R}", graph=layered_graph(16, 16, 1), R=R,
                betas=geometric_betas(R, 0.1, 3.0), seed=5489, field_bits=16, sweeps=500,
                swap_every=0)


def config_paper():
    """The paper's workload shape (section 4): 256 Trotter layers of 96 spins
    (an 8 x 12 lattice plus matchings; 24576 spins, degree 6-8), 115 models
    (replicas) at geometric betas 0.1..3.0, 30000 sweeps, no PT in the timing.
    The paper's 115 QMC models are not available; this synthetic model of the
    same shape stands in for them."""
    return dict(name="paper_96x256_R115", graph=layered_graph(8, 256, 1, Ly=12), R=115,
                betas=geometric_betas(115, 0.1, 3.0), seed=5489, field_bits=16, sweeps=30000,
                swap_every=0)


def ragged_instances(n_inst: int = 4096, batch_seed: int = 2024):
    """Descriptors of the ragged batch: spin counts log-uniform in 2^11..2^15.

    log2 N ~ U[11, 15], M in {16, 32}, L = clamp(round(sqrt(N/M)), 8, 32),
    R ~ U{8..64}; instance b uses graph_seed 1000 + b and seed 5489 + 1000 b,
    betas geometric 0.1..3.0.  Graph construction is deferred (``build_instance``)
    because 4096 graphs take a while in Python; identical (L, graph_seed) pairs
    are cached.
    """
    rng = np.random.default_rng(batch_seed)
    out = []
    for b in range(n_inst):
        lg = rng.uniform(11.0, 15.0)
        M = int(rng.choice([16, 32]))
        L = int(min(32, max(8, round(np.sqrt(2.0 ** lg / M)))))
        R = int(rng.integers(8, 65))
        out.append(dict(index=b, L=L, M=M, R=R, graph_seed=1000 + b, seed=5489 + 1000 * b))
    return out


def build_instance(desc) -> dict:
    g = layered_graph(desc["L"], desc["M"], desc["graph_seed"])
    return dict(graph=g, R=desc["R"], betas=geometric_betas(desc["R"], 0.1, 3.0),
                seed=desc["seed"])
