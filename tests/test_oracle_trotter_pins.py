"""Pins of the oracle's split-coupling mode (no GPU).

The layered models of section 4 come from a Trotter decomposition whose
inter-slice coupling depends on the temperature.  With split couplings the
oracle weights a state at temperature k by exp(-beta_k E_space - K_k C),
E_space the cost function over in-slice edges and C = -sum over Trotter
(inter-slice) pairs of s s'.  These tests fix that rule from outside the
oracle: the deterministic exponential against 40-digit arithmetic, exact
transition matrices built here from the definition, histograms of the
oracle's chains against exact Boltzmann enumeration, closed-form energy and
field decompositions, and bit-exact agreement with the plain mode where the
two rules coincide.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1004_0024_gb300 import workloads as W

TOP = 2**32 - 1


def _tiny_layered(S_edges, h, S, M, ring=True, j_tau=4):
    """M copies of one slice (S sites, edges {(a, b): J}, fields h) joined by
    Trotter pairs (t S + q, (t + 1) S + q): a ring for M >= 3, else a chain."""
    edges = {}
    for t in range(M):
        for (a, b), j in S_edges.items():
            edges[(t * S + a, t * S + b)] = j
    last = M if ring else M - 1
    for t in range(last):
        for q in range(S):
            a, b = t * S + q, ((t + 1) % M) * S + q
            edges[(min(a, b), max(a, b))] = j_tau
    return W.graph_from_edges(S * M, edges, np.tile(np.asarray(h), M), n_slices=M)


def _states(n):
    x = np.arange(2**n)
    return np.where((x[:, None] >> np.arange(n)) & 1, 1, -1)


def _parts(g):
    """Spatial and Trotter edge lists [(i, j, J)] (each pair once)."""
    S = g.slice_size
    sp, tr = [], []
    for i in range(g.n):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            j = int(g.col[e])
            if j > i:
                (sp if i // S == j // S else tr).append((i, j, int(g.J[e])))
    return sp, tr


def _e_space(g, s, sp):
    return -int(np.dot(g.h, s)) - sum(J * int(s[i]) * int(s[j]) for i, j, J in sp)


def _c_trotter(s, tr):
    return -sum(int(s[i]) * int(s[j]) for i, j, _ in tr)


def _threshold(p):
    return min(math.floor(math.ldexp(p, 32)), TOP)


def _accept_prob(z, expfn):
    """Probability of the rule: T = 2^32 - 1 for z <= 0, else
    min(floor(2^32 e^-z), 2^32 - 1); T = 2^32 - 1 accepts every word, any
    other T accepts the T words below it."""
    t = TOP if z <= 0 else _threshold(expfn(-z))
    return 1.0 if t == TOP else t / 2**32


def _split_sweep_matrix(g, beta, K, order, sign=1):
    """One sweep as the product of single-spin kernels under split couplings:
    z = 2 (beta s f_space + K s tau) and the acceptance of ``_accept_prob``
    with libm's exp.  ``sign = -1`` flips the Trotter term (a wrong rule the
    histogram test must reject)."""
    n, S = g.n, g.slice_size
    X = _states(n)
    P = np.eye(2**n)
    for i in order:
        Ki = np.zeros((2**n, 2**n))
        lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
        nb, Jn = g.col[lo:hi], g.J[lo:hi]
        spatial = nb // S == i // S
        for x in range(2**n):
            s = X[x]
            ks = int(s[i]) * (int(g.h[i]) + int(np.dot(Jn[spatial], s[nb[spatial]])))
            kt = sign * int(s[i]) * int(s[nb[~spatial]].sum())
            z = 2.0 * (beta * ks + K * kt)
            a = _accept_prob(z, math.exp)
            Ki[x, x ^ (1 << i)] += a
            Ki[x, x] += 1 - a
        P = P @ Ki
    return P


def _boltzmann(g, beta, K):
    sp, tr = _parts(g)
    X = _states(g.n)
    w = np.array([-beta * _e_space(g, s, sp) - K * _c_trotter(s, tr) for s in X])
    p = np.exp(w - w.max())
    return p / p.sum()


# ---------------------------------------------------- deterministic exp
def test_deterministic_exp_is_within_one_ulp_of_exp():
    """Cody-Waite reduction plus a degree-13 Taylor polynomial: within 1.5 ulp
    of e^x (40-digit reference) over [-708, 0] and near 0, exact at 0, 0 below
    -708, and monotone on a fine grid of the swap rule's range."""
    import mpmath
    mpmath.mp.dps = 40
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-708, 0, 3000), rng.uniform(-1, 0, 1000),
                         -np.logspace(-18, 2.8, 600), [-0.5 * math.log(2), -math.log(2)]])
    worst = 0.0
    for x in xs.tolist():
        v = oracle.exp_det(x)
        err = abs(mpmath.mpf(v) - mpmath.exp(mpmath.mpf(x))) / math.ulp(v)
        worst = max(worst, float(err))
    assert worst <= 1.5
    assert oracle.exp_det(0.0) == 1.0 and oracle.exp_det(-1e-300) == 1.0
    assert oracle.exp_det(-708.5) == 0.0 and oracle.exp_det(-1e6) == 0.0
    grid = np.linspace(-25.0, 0.0, 20001).tolist()
    vals = [oracle.exp_det(x) for x in grid]
    assert all(a <= b for a, b in zip(vals, vals[1:]))


def test_split_thresholds_follow_their_definitions():
    """floor(2^32 e^-z) for z > 0 (libm exp for flips, the deterministic one
    for swaps), each product of z rounded on its own; z <= 0 has none."""
    import mpmath
    mpmath.mp.dps = 50
    for beta, K in [(0.3, 0.8), (1.7, 0.05), (0.05, 2.5)]:
        for ks in range(-6, 7):
            for kt in (-2, 0, 2):
                z = 2.0 * (beta * ks + K * kt)
                got = oracle.trotter_flip_threshold(beta, K, ks, kt)
                if z <= 0:
                    assert got == TOP
                    continue
                exact = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-mpmath.mpf(z)), 32)))
                assert abs(got - min(exact, TOP)) <= 1
    for dbeta, dK in [(0.02, -0.1), (0.3, 0.05), (1e-3, -2.0)]:
        for dE in (-40, -3, 0, 1, 17, 250):
            for dC in (-12, -2, 0, 4, 30):
                z = dbeta * dE + dK * dC
                got = oracle.trotter_swap_threshold(dbeta, dK, dE, dC)
                if z <= 0:
                    assert got == TOP
                    continue
                exact = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-mpmath.mpf(z)), 32)))
                assert abs(got - min(exact, TOP)) <= 1


# ---------------------------------------------- energy decomposition
def test_split_state_decomposes_the_plain_energy_and_fields():
    """On a layered model with uniform Trotter coupling j_tau the plain cost
    function is E_space + j_tau C and the plain field f_space + j_tau tau;
    the split chain keeps f_space, E_space and C equal to their definitions
    through sweeps and swaps."""
    g = W.layered_graph(3, 5, graph_seed=11, j_tau=4)
    betas = W.geometric_betas(6, 0.2, 1.5)
    K = 0.5 * np.log(1.0 / np.tanh(betas * 1.5 / 5))
    sim = oracle.Sim(g, betas, seed=77, rng="philox", threads=1)
    sim.set_trotter(K)
    sp, tr = _parts(g)
    S = g.slice_size
    for _ in range(6):
        sim.run(5, 1)
        st = sim.read()
        C = sim.read_trotter()
        for r in range(sim.R):
            s = st["spins"][r]
            assert st["energy"][r] == _e_space(g, s, sp)
            assert C[r] == _c_trotter(s, tr)
            assert oracle.energy(g, s) == st["energy"][r] + 4 * C[r]
            f_plain = oracle.fields(g, s)
            rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
            cross = rows // S != g.col // S
            tau = np.bincount(rows[cross], weights=s[g.col[cross]], minlength=g.n).astype(np.int64)
            assert np.array_equal(st["fields"][r], f_plain - 4 * tau)
    assert st["sweeps"] == 30 and st["passes"] == 30


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_split_mode_reproduces_the_plain_chain_where_the_rules_coincide(rng):
    """With K_k = beta_k j_tau and dyadic temperatures every exponent is the
    same FP64 number in both modes, so the split chain (sweeps and PT) is the
    plain chain bit for bit: spins, labels and acceptance counts."""
    g = W.layered_graph(3, 4, graph_seed=5, j_tau=4)
    betas = np.array([0.125, 0.25, 0.375, 0.5, 0.75])
    plain = oracle.Sim(g, betas, seed=1234, rng=rng, threads=1)
    split = oracle.Sim(g, betas, seed=1234, rng=rng, threads=1)
    split.set_trotter(4.0 * betas)
    plain.run(40, 1)
    split.run(40, 1)
    a, b = plain.read(), split.read()
    assert np.array_equal(a["spins"], b["spins"])
    assert np.array_equal(a["temp_of_slot"], b["temp_of_slot"])
    assert np.array_equal(a["swap_acc"], b["swap_acc"]) and a["swap_acc"].sum() > 0
    assert np.array_equal(a["energy"], b["energy"] + 4 * split.read_trotter())


# ---------------------------------------------- exact kernels and chains
def test_split_sweep_leaves_the_split_boltzmann_law_stationary():
    """pi P = pi for the sequential sweep under split couplings with K
    unrelated to beta (residual only from the 2^-32 truncation); the plain
    law exp(-beta (E_space + j_tau C)) is not stationary for it."""
    g = _tiny_layered({(0, 1): -2}, [1, -1], S=2, M=4)
    beta, K = 0.45, 0.8
    P = _split_sweep_matrix(g, beta, K, range(g.n))
    pi = _boltzmann(g, beta, K)
    assert np.allclose(P.sum(1), 1.0)
    assert np.abs(pi @ P - pi).max() < 1e-8
    wrong = _boltzmann(g, beta, 4 * beta)
    assert np.abs(wrong @ P - wrong).max() > 1e-3


def test_split_one_sweep_outcomes_match_the_exact_row():
    """40000 replicas start at one state and take one oracle sweep under
    split couplings: the outcome histogram fits the exact row and rejects the
    row with the Trotter term's sign flipped."""
    g = _tiny_layered({(0, 1): 2}, [1, 0], S=2, M=3)
    beta, K, R = 0.35, 0.6, 40000
    x0 = 0b101101
    s0 = _states(g.n)[x0]
    sim = oracle.Sim(g, [beta] * R, seed=2718, threads=1)
    sim.set_trotter([K] * R)
    sim.set_spins(s0)
    sim.sweep(1)
    out = sim.read()["spins"]
    idx = ((out > 0).astype(np.int64) << np.arange(g.n)).sum(1)
    counts = np.bincount(idx, minlength=2**g.n)
    row = _split_sweep_matrix(g, beta, K, range(g.n))[x0]
    bad = _split_sweep_matrix(g, beta, K, range(g.n), sign=-1)[x0]
    assert np.abs(row - bad).sum() > 0.1

    def pval(p):
        m = p * R >= 5
        obs = np.append(counts[m], counts[~m].sum())
        exp = np.append(p[m] * R, p[~m].sum() * R)
        keep = exp > 0
        return stats.chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum()).pvalue

    assert pval(row) > 1e-3
    assert pval(bad) < 1e-6


def test_split_pt_joint_chain_is_stationary():
    """Exact matrix of (sweep both replicas; one swap) on a 2-slice chain of
    2 sites: the product of the two split Boltzmann laws is invariant when the
    swap uses z = dbeta dE + dK dC with the deterministic exponential, and
    not when the dK dC term is dropped."""
    g = _tiny_layered({(0, 1): 1}, [2, -1], S=2, M=2, ring=False)
    (b0, K0), (b1, K1) = (0.3, 1.1), (0.7, 0.4)
    sp, tr = _parts(g)
    X = _states(g.n)
    E = np.array([_e_space(g, s, sp) for s in X])
    C = np.array([_c_trotter(s, tr) for s in X])
    ns = 2**g.n
    sweep = np.kron(_split_sweep_matrix(g, b0, K0, range(g.n)),
                    _split_sweep_matrix(g, b1, K1, range(g.n)))
    pi = np.outer(_boltzmann(g, b0, K0), _boltzmann(g, b1, K1)).ravel()

    def swap_matrix(with_c):
        Q = np.zeros((ns * ns, ns * ns))
        for x in range(ns):
            for y in range(ns):
                z = (b1 - b0) * int(E[x] - E[y]) + ((K1 - K0) * int(C[x] - C[y]) if with_c else 0.0)
                a = _accept_prob(z, oracle.exp_det)
                Q[x * ns + y, y * ns + x] += a
                Q[x * ns + y, x * ns + y] += 1 - a
        return Q

    assert np.abs(pi @ (sweep @ swap_matrix(True)) - pi).max() < 1e-8
    assert np.abs(pi @ (sweep @ swap_matrix(False)) - pi).max() > 1e-4


def test_split_pt_chain_matches_boltzmann_at_every_temperature():
    """8 spins (2 sites x 4 slices), 3 temperatures with K_k falling as
    beta_k rises, PT after every sweep: the state found at each temperature
    index follows exp(-beta_k E_space - K_k C) (chi-square over 256 states)."""
    g = _tiny_layered({(0, 1): -1}, [1, 1], S=2, M=4)
    betas = np.array([0.15, 0.3, 0.5])
    K = 0.5 * np.log(1.0 / np.tanh(betas * 2.0 / 4))
    sim = oracle.Sim(g, betas, seed=99, threads=1)
    sim.set_trotter(K)
    sim.run(200, 1)
    weights = 1 << np.arange(g.n)
    nsamp = 12000
    counts = np.zeros((3, 2**g.n), dtype=np.int64)
    for _ in range(nsamp):
        sim.run(6, 1)
        st = sim.read()
        idx = ((st["spins"] > 0).astype(np.int64) * weights).sum(1)
        for k in range(3):
            counts[k, idx[np.where(st["temp_of_slot"] == k)[0][0]]] += 1
    for k in range(3):
        p = _boltzmann(g, betas[k], K[k])
        m = p * nsamp >= 5
        obs, exp = counts[k][m], p[m] * nsamp
        if (~m).any():
            obs, exp = np.append(obs, counts[k][~m].sum()), np.append(exp, p[~m].sum() * nsamp)
        assert stats.chisquare(obs, exp * obs.sum() / exp.sum()).pvalue > 1e-4, k
    assert sim.read()["swap_acc"].min() > 0
