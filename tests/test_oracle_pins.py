"""Pins of the oracle against facts fixed by the paper and by mathematics (no GPU).

Each test names what it pins.  The oracle is only trusted as a parity
reference because these pass: known RNG outputs, closed-form energies and
fields, exact transition matrices of the sequential sweep, Boltzmann
enumeration of long chains with parallel tempering, and deterministic special
cases (all-zero model, frozen chains, isolated spins, strict comparison).
"""
from __future__ import annotations

import math

import numpy as np
import pytest
from scipy import stats

import oracle
from conftest import golden_path
from paper_1004_0024_gb300 import workloads as W


def _golden_rows(name):
    rows = []
    with open(golden_path(name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ RNGs
def test_mt19937_known_outputs():
    """init_genrand(5489): first output 3499211612, 10000th 4123659995."""
    for seed, idx, val in _golden_rows("mt19937_known.txt"):
        out = oracle.mt_stream(int(seed), int(idx))
        assert int(out[int(idx) - 1]) == int(val)


@pytest.mark.parametrize("seed", [0, 1, 42, 5489, 5489 + 255, 2**32 - 1])
def test_mt19937_matches_numpy_legacy_generator(seed):
    """numpy's legacy RandomState(seed) is MT19937 under init_genrand(seed)."""
    ref = np.random.RandomState(seed)._bit_generator.random_raw(3000).astype(np.uint32)
    assert np.array_equal(oracle.mt_stream(seed, 3000), ref)


def test_philox4x32_10_known_answers():
    for row in _golden_rows("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        assert list(oracle.philox(vals[0:4], vals[4:6])) == vals[6:10]


# ------------------------------------------------------------ thresholds
def _exact_floor(expr_digits: str) -> int:
    import mpmath
    return int(mpmath.floor(mpmath.mpf(expr_digits)))


@pytest.mark.parametrize("beta", [0.05, 0.1, 0.37, 1.0, 3.0, 5.0])
def test_flip_threshold_is_floor_2p32_exp_minus_2beta_k(beta):
    """T_beta(k) = floor(2^32 exp(-2 beta k)) (Metropolis, dE = 2k); checked at
    60 digits, off by at most one unit from FP64 rounding, and decreasing."""
    import mpmath
    mpmath.mp.dps = 60
    prev = 2**32
    for k in range(1, 40):
        exact = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-2 * mpmath.mpf(beta) * k), 32)))
        got = oracle.flip_threshold(beta, k)
        assert abs(got - exact) <= 1
        assert got <= prev
        prev = got
    # the factor 2: exp(-2 beta) vs exp(-beta) differ widely at k = 1
    assert oracle.flip_threshold(beta, 1) < math.ldexp(math.exp(-beta), 32) - 1


@pytest.mark.parametrize("dbeta", [1e-3, 0.02, 0.3])
def test_swap_threshold_is_floor_2p32_exp_minus_dbeta_d(dbeta):
    import mpmath
    mpmath.mp.dps = 60
    for d in (1, 2, 7, 50, 400):
        exact = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-mpmath.mpf(dbeta) * d), 32)))
        assert abs(oracle.swap_threshold(dbeta, d) - exact) <= 1


# ------------------------------------------------------ energy and fields
def test_energy_and_fields_closed_forms():
    """Section 1 cost function, each edge counted once; f_i = h_i + sum_j J_ij s_j."""
    tri = W.graph_from_edges(3, {(0, 1): 1, (1, 2): 1, (0, 2): 1}, [0, 0, 0])
    assert oracle.energy(tri, np.array([1, 1, 1])) == -3
    assert oracle.energy(tri, np.array([1, 1, -1])) == 1
    assert list(oracle.fields(tri, np.array([1, 1, -1]))) == [0, 0, 2]
    g = W.graph_from_edges(4, {(0, 1): -2, (1, 2): 3, (2, 3): 1, (0, 3): -1}, [1, -2, 0, 2])
    s = np.array([1, -1, -1, 1])
    # -sum h s = -(1 + 2 + 0 + 2) = -5 ; -sum J s s = -(2 + 3 - 1 - 1) = -3
    assert oracle.energy(g, s) == -8
    assert list(oracle.fields(g, s)) == [1 + 2 - 1, -2 - 2 - 3, 0 - 3 + 1, 2 - 1 - 1]


# -------------------------------------------------------- special cases
def test_zero_model_flips_every_spin_every_sweep():
    """h = J = 0 gives k = 0 everywhere, so every visit flips (k <= 0 rule)."""
    g = W.graph_from_edges(37, {}, np.zeros(37))
    sim = oracle.Sim(g, [0.5, 1.0], seed=11)
    s0 = sim.read()["spins"]
    sim.sweep(1)
    assert np.array_equal(sim.read()["spins"], -s0)
    sim.sweep(1)
    st = sim.read()
    assert np.array_equal(st["spins"], s0) and (st["energy"] == 0).all()


def test_isolated_spins_field_equals_h():
    h = np.array([3, -2, 0, 1, -1, 2])
    g = W.graph_from_edges(6, {}, h)
    sim = oracle.Sim(g, [0.3], seed=3)
    sim.sweep(3)
    st = sim.read()
    assert np.array_equal(st["fields"][0], h)
    assert st["energy"][0] == -int(np.dot(h, st["spins"][0]))


def test_frozen_chain_is_greedy_descent():
    """At beta = 200 every T(k >= 1) is 0, so only k <= 0 moves are taken: the
    sweep is the deterministic sequential descent, replayed here by hand."""
    g = W.random_graph(24, 50, seed=5)
    sim = oracle.Sim(g, [200.0, 200.0], seed=9)
    assert oracle.flip_threshold(200.0, 1) == 0
    st = sim.read()
    s = st["spins"].astype(np.int64).copy()
    sim.sweep(4)
    for r in range(2):
        for _ in range(4):
            for i in range(g.n):
                lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
                f = g.h[i] + int(np.dot(g.J[lo:hi], s[r, g.col[lo:hi]]))
                if s[r, i] * f <= 0:
                    s[r, i] = -s[r, i]
    assert np.array_equal(sim.read()["spins"], s)


def test_strict_comparison_and_first_sweep_word():
    """One spin, h = 1: the initial spin is +1 (bit 31 of the first MT word of
    seed 5489 is set), so k = 1 and the first sweep draws the SECOND word u.
    With T(1) == u exactly the flip is refused (u < T is strict, Figure 1);
    with T(1) == u + 1 it is taken."""
    u = int(oracle.mt_stream(5489, 2)[1])
    g = W.graph_from_edges(1, {}, [1])

    def beta_for(target):
        b = -math.log((target + 0.5) / 2**32) / 2
        assert oracle.flip_threshold(b, 1) == target
        return b

    assert oracle.mt_stream(5489, 1)[0] >> 31 == 1
    sim = oracle.Sim(g, [beta_for(u)], seed=5489)
    assert sim.read()["spins"][0, 0] == 1
    sim.sweep(1)
    assert sim.read()["spins"][0, 0] == 1
    sim = oracle.Sim(g, [beta_for(u + 1)], seed=5489)
    sim.sweep(1)
    assert sim.read()["spins"][0, 0] == -1


# --------------------------------------------- RNG consumption / counter maps
@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_word_map_per_spin(rng):
    """Isolated spins with h = 1 reveal every word: an up spin (k = 1) flips iff
    u < T(1), a down spin (k = -1) always flips.  The prediction uses the
    documented stream positions / counter map, not the oracle's sweep code."""
    S, M, R, seed, inst, beta = 6, 5, 3, 77, 9, 0.35
    n = S * M
    g = W.graph_from_edges(n, {}, np.ones(n))
    g.n_slices = M
    T1 = oracle.flip_threshold(beta, 1)
    sim = oracle.Sim(g, [beta] * R, seed=seed, rng=rng, instance=inst)

    def word(r, i, c, tag):
        if rng == "mt19937":
            pos = i if tag == 3 else n * (1 + c) + i
            return int(oracle.mt_stream(seed + r, pos + 1)[pos])
        t, q = divmod(i, S)
        return int(oracle.philox([(t >> 2) * S + q, c if tag == 0 else 0, inst, tag],
                                 [seed, r])[t & 3])

    s = np.array([[1 if word(r, i, 0, 3) >> 31 else -1 for i in range(n)] for r in range(R)])
    assert np.array_equal(sim.read()["spins"], s)
    for c in range(3):
        for r in range(R):
            for i in range(n):
                if s[r, i] < 0 or word(r, i, c, 0) < T1:
                    s[r, i] = -s[r, i]
        sim.sweep(1)
        assert np.array_equal(sim.read()["spins"], s)


@pytest.mark.parametrize("rng", ["mt19937", "philox"])
def test_pt_schedule_words_and_rule_on_frozen_energies(rng):
    """No sweeps between passes, so energies stay put and every decision is
    predicted from the pass parity, the swap-stream word and the rule
    accept iff d <= 0 or u < floor(2^32 exp(-(b_{k+1}-b_k) d))."""
    R, seed, inst = 7, 1234, 5
    h = np.array([3, -2, 1, 2, -1, 3, -3, 2, 1, -2])
    g = W.graph_from_edges(h.size, {}, h)
    betas = W.geometric_betas(R, 0.02, 0.6)
    sim = oracle.Sim(g, betas, seed=seed, rng=rng, instance=inst)
    E = sim.read()["energy"].copy()
    assert len(set(E.tolist())) > 3
    slot_of_temp = list(range(R))
    mt = oracle.mt_stream(seed + R, 4000)
    pos = 0
    for p in range(60):
        for k in range(p % 2, R - 1, 2):
            if rng == "mt19937":
                u = int(mt[pos]); pos += 1
            else:
                j = k >> 1
                u = int(oracle.philox([j >> 2, p, inst, 1], [seed, 0xFFFFFFFF])[j & 3])
            a, b = slot_of_temp[k], slot_of_temp[k + 1]
            d = int(E[a] - E[b])
            thr = math.floor(math.ldexp(math.exp(-(betas[k + 1] - betas[k]) * d), 32)) if d > 0 else None
            if d <= 0 or u < thr:
                slot_of_temp[k], slot_of_temp[k + 1] = b, a
        sim.pt_swap()
        temp = sim.read()["temp_of_slot"]
        assert [int(np.where(temp == k)[0][0]) for k in range(R)] == slot_of_temp


def test_pt_always_accepts_at_equal_energy_and_alternates_parity():
    """h = J = 0: every energy is 0, d = 0 always accepts; pass p swaps the
    pairs (k, k+1) with k = p mod 2, so the labels move as a brick pattern."""
    R = 6
    g = W.graph_from_edges(5, {}, np.zeros(5))
    sim = oracle.Sim(g, W.geometric_betas(R, 0.1, 1.0), seed=2)
    slot_of_temp = list(range(R))
    for p in range(9):
        for k in range(p % 2, R - 1, 2):
            slot_of_temp[k], slot_of_temp[k + 1] = slot_of_temp[k + 1], slot_of_temp[k]
        sim.pt_swap()
        st = sim.read()
        assert [int(np.where(st["temp_of_slot"] == k)[0][0]) for k in range(R)] == slot_of_temp
    assert st["passes"] == 9
    assert list(st["swap_acc"]) == [5, 4, 5, 4, 5]


# ------------------------------------------ exact sequential-sweep kernel
def _states(n):
    x = np.arange(2**n)
    return np.where((x[:, None] >> np.arange(n)) & 1, 1, -1)


def _energies(g, S):
    return np.array([oracle.energy(g, s) for s in S])


def _sweep_matrix(g, beta, order):
    """One sweep as the product of single-spin Metropolis kernels K_i in the
    given visit order, with acceptance T(k)/2^32 (k <= 0: 1)."""
    n = g.n
    S = _states(n)
    P = np.eye(2**n)
    for i in order:
        K = np.zeros((2**n, 2**n))
        for x in range(2**n):
            s = S[x]
            lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
            f = int(g.h[i]) + int(np.dot(g.J[lo:hi], s[g.col[lo:hi]]))
            k = int(s[i]) * f
            a = 1.0 if k <= 0 else math.floor(math.ldexp(math.exp(-2 * beta * k), 32)) / 2**32
            K[x, x ^ (1 << i)] += a
            K[x, x] += 1 - a
        P = P @ K
    return P


def test_sequential_sweep_leaves_boltzmann_stationary():
    """pi P = pi for the sequential Metropolis sweep with integer thresholds;
    the residual comes only from the 2^-32 truncation of T."""
    g = W.random_graph(6, 9, seed=21)
    beta = 0.45
    P = _sweep_matrix(g, beta, range(g.n))
    E = _energies(g, _states(g.n))
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    assert np.abs(pi @ P - pi).max() < 1e-8
    assert np.allclose(P.sum(1), 1.0)


def test_one_sweep_outcome_distribution_matches_exact_row():
    """Start 40000 independent replicas at the same state x0, take one oracle
    sweep, and compare the outcome histogram with row x0 of the exact
    sequential-order matrix (a reversed visit order is clearly rejected)."""
    g = W.random_graph(5, 7, seed=8)
    beta, R = 0.3, 40000
    x0 = 0b10110
    s0 = _states(g.n)[x0]
    sim = oracle.Sim(g, [beta] * R, seed=99)
    sim.set_spins(s0)
    sim.sweep(1)
    out = sim.read()["spins"]
    idx = ((out > 0).astype(np.int64) << np.arange(g.n)).sum(1)
    counts = np.bincount(idx, minlength=2**g.n)
    row = _sweep_matrix(g, beta, range(g.n))[x0]
    rev = _sweep_matrix(g, beta, range(g.n - 1, -1, -1))[x0]
    assert np.abs(row - rev).sum() > 0.1  # the test can tell the orders apart

    def pval(p):
        m = p * R >= 5
        obs = np.append(counts[m], counts[~m].sum())
        exp = np.append(p[m] * R, p[~m].sum() * R)
        keep = exp > 0
        return stats.chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum()).pvalue

    assert pval(row) > 1e-3
    assert pval(rev) < 1e-6


def test_long_pt_chain_matches_boltzmann_at_every_temperature():
    """8 spins, 4 temperatures, PT after every sweep: the state found at each
    temperature index follows exp(-beta_k E) (chi-square over all 256 states)."""
    g = W.random_graph(8, 12, seed=4, jmax=2)
    betas = np.array([0.1, 0.2, 0.3, 0.45])
    sim = oracle.Sim(g, betas, seed=314)
    sim.run(200, 1)
    S = _states(g.n)
    E = _energies(g, S)
    weights = (1 << np.arange(g.n))
    counts = np.zeros((4, 2**g.n), dtype=np.int64)
    nsamp = 12000
    for _ in range(nsamp):
        sim.run(8, 1)
        st = sim.read()
        idx = ((st["spins"] > 0).astype(np.int64) * weights).sum(1)
        for k in range(4):
            counts[k, idx[np.where(st["temp_of_slot"] == k)[0][0]]] += 1
    for k, b in enumerate(betas):
        p = np.exp(-b * (E - E.min()))
        p /= p.sum()
        m = p * nsamp >= 5
        obs, exp = counts[k][m], p[m] * nsamp
        if (~m).any():
            obs, exp = np.append(obs, counts[k][~m].sum()), np.append(exp, p[~m].sum() * nsamp)
        assert stats.chisquare(obs, exp * obs.sum() / exp.sum()).pvalue > 1e-4, k
    assert sim.read()["swap_acc"].min() > 0


def test_pt_joint_chain_product_boltzmann_is_stationary():
    """Exact matrix of (sweep both replicas; one PT pass) on 3 spins x 2
    temperatures x 2 label assignments: the product Boltzmann law is invariant."""
    g = W.random_graph(3, 3, seed=2)
    b0, b1 = 0.3, 0.8
    n = g.n
    E = _energies(g, _states(n))
    P0, P1 = _sweep_matrix(g, b0, range(n)), _sweep_matrix(g, b1, range(n))
    ns = 2**n
    # joint state (x_at_b0, x_at_b1); the label swap exchanges the two states
    sweep = np.kron(P0, P1)
    swap = np.zeros((ns * ns, ns * ns))
    for x in range(ns):
        for y in range(ns):
            d = E[x] - E[y]
            a = 1.0 if d <= 0 else math.floor(math.ldexp(math.exp(-(b1 - b0) * d), 32)) / 2**32
            swap[x * ns + y, y * ns + x] += a
            swap[x * ns + y, x * ns + y] += 1 - a
    P = sweep @ swap
    pi = np.outer(np.exp(-b0 * (E - E.min())), np.exp(-b1 * (E - E.min()))).ravel()
    pi /= pi.sum()
    assert np.abs(pi @ P - pi).max() < 1e-8


# --------------------------------------------------- invariants on cfg0
def test_oracle_invariants_on_layered_config():
    c = W.config0()
    g = c["graph"]
    assert set(np.unique(g.degrees)) <= {6, 7, 8}
    sim = oracle.Sim(g, c["betas"], c["seed"])
    sim.run(40, 1)
    st = sim.read()
    for r in range(c["R"]):
        assert np.array_equal(oracle.fields(g, st["spins"][r]), st["fields"][r])
        assert oracle.energy(g, st["spins"][r]) == st["energy"][r]
    assert sorted(st["temp_of_slot"].tolist()) == list(range(c["R"]))
    assert st["sweeps"] == 40 and st["passes"] == 40


# ---------------------------------------------- exp approximations (section 2.4)
def _exp_approx_grid(lo, hi, n, accurate):
    ys = np.linspace(lo, hi, n, endpoint=False)
    xs = ys * np.log(2.0)
    approx = np.array([oracle.exp_approx(float(x), accurate) for x in xs])
    exact = np.exp(xs.astype(np.float32).astype(np.float64))
    return ys, approx, exact


def test_fast_exp_approximation_has_the_papers_error_figures():
    """Unscaled, the fast approximation interpolates 2^y linearly between
    integer y (exact there) with mean relative error (2 ln^2 2)^-1 - 1 =
    0.0407 (Appendix); the 2 ln^2 2 factor brings the mean to zero."""
    scale = 2.0 * np.log(2.0) ** 2
    for n in range(-20, 1):
        assert oracle.exp_approx(n * np.log(2.0)) / np.float32(scale) == pytest.approx(2.0 ** n, rel=1e-6)
    ys, approx, exact = _exp_approx_grid(-6.0, 0.0, 24000, False)
    rel_unscaled = approx / np.float32(scale) / exact - 1.0
    assert abs(rel_unscaled.mean() - (1.0 / scale - 1.0)) < 5e-4
    assert abs(1.0 / scale - 1.0 - 0.0407) < 1e-4
    assert abs((approx / exact - 1.0).mean()) < 5e-4
    assert oracle.exp_approx(-127.0 * np.log(2.0)) == 0.0  # below -126 ln 2


def test_accurate_exp_approximation_stays_in_the_papers_band():
    """The accurate approximation (2^(4y) interpolated, fourth root taken
    exactly) has relative error within (-0.01, 0.005) over its range
    -31.5 <= y < 0, and is 0 below it (Appendix, Figure 17)."""
    ys, approx, exact = _exp_approx_grid(-31.5, 0.0, 20000, True)
    rel = approx / exact - 1.0
    assert rel.min() > -0.01 and rel.max() < 0.005, (rel.min(), rel.max())
    assert oracle.exp_approx(-32.0 * np.log(2.0), True) == 0.0


@pytest.mark.parametrize("mode", ["fast", "accurate"])
def test_approximate_flip_thresholds_are_monotone_and_close(mode):
    """Thresholds built with an approximate exponential decrease with k, and
    stay within the approximation's error of the exact ones."""
    band = 0.045 if mode == "fast" else 0.011
    for beta in (0.1, 0.7, 2.5):
        prev = 2 ** 32
        for k in range(1, 60):
            t = oracle.flip_threshold_mode(beta, k, mode)
            assert t <= prev
            prev = t
            ex = oracle.flip_threshold(beta, k)
            if ex > 1 << 12:
                assert abs(t / ex - 1.0) < band, (beta, k, t, ex)
