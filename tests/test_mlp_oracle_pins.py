"""Pins of the learned-proposal oracle (no GPU): backpropagation against finite
differences, the column energy against the full cost function, the proposal's
normalisation, and exact stationarity of the column Metropolis-Hastings move."""
import itertools
import math

import numpy as np

import oracle
from paper_1004_0024_gb300 import workloads as W


def _net(IN=33, H=16, OUT=8, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.normal(0, 0.4, (H, IN)), rng.normal(0, 0.1, H), rng.normal(0, 0.3, (H, H)),
            rng.normal(0, 0.1, H), rng.normal(0, 0.3, (OUT, H)), rng.normal(0, 0.1, OUT)]


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(1)
    net = _net()
    X = rng.normal(0, 1, (5, 33))
    Y = (rng.random((5, 8)) < 0.5).astype(float)
    loss, grads = oracle.mlp_backward(X, Y, *net)
    for li, (w, g) in enumerate(zip(net, grads)):
        flat = w.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            eps = 1e-6
            flat[idx] = old + eps
            lp, _ = oracle.mlp_backward(X, Y, *net)
            flat[idx] = old - eps
            lm, _ = oracle.mlp_backward(X, Y, *net)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g.reshape(-1)[idx]) <= 1e-6 + 1e-5 * abs(fd), (li, idx)


def test_forward_is_relu_mlp():
    net = _net(IN=3, H=4, OUT=2, seed=3)
    X = np.array([[0.5, -1.0, 2.0]])
    H1, H2, L = oracle.mlp_forward(X, *net)
    h1 = np.maximum(net[0] @ X[0] + net[1], 0)
    h2 = np.maximum(net[2] @ h1 + net[3], 0)
    assert np.allclose(H1[0], h1) and np.allclose(H2[0], h2)
    assert np.allclose(L[0], net[4] @ h2 + net[5])


def test_column_energy_is_the_cost_function_difference():
    """E(full model with column s') - E(... s) equals E_col(s') - E_col(s)."""
    g = W.layered_graph(4, 5, graph_seed=3, j_tau=3)
    S, M = 16, 5
    rng = np.random.default_rng(2)
    s = rng.choice([-1, 1], size=g.n).astype(np.int8)
    for q in (0, 7, 15):
        idx = np.arange(M) * S + q
        col = s[idx].copy()
        f = oracle.fields(g, s)
        phi = f[idx] - 3 * (np.roll(col, 1) + np.roll(col, -1))
        new = rng.choice([-1, 1], size=M).astype(np.int8)
        s2 = s.copy()
        s2[idx] = new
        d_full = oracle.energy(g, s2) - oracle.energy(g, s)
        d_col = oracle.column_energy(M, 3, phi, new) - oracle.column_energy(M, 3, phi, col)
        assert d_full == d_col


def test_proposal_is_normalised():
    lg = np.array([0.3, -1.2, 2.0, 0.0])
    tot = sum(math.exp(oracle.log_q(lg, np.array(c, np.int8)))
              for c in itertools.product([-1, 1], repeat=4))
    assert abs(tot - 1.0) < 1e-12


def test_column_move_leaves_conditional_boltzmann_stationary():
    """Exact 2^M x 2^M matrix of one MH column move with a fixed arbitrary
    proposal: the conditional law exp(-beta E_col) is invariant."""
    M, jtau, beta = 4, 2, 0.7
    phi = np.array([3, -1, 0, 2], np.int32)
    lg = np.array([0.4, -0.9, 1.3, 0.2])
    cols = [np.array(c, np.int8) for c in itertools.product([-1, 1], repeat=M)]
    n = len(cols)
    P = np.zeros((n, n))
    for a, s in enumerate(cols):
        for b, s2 in enumerate(cols):
            if a == b:
                continue
            la, _ = oracle.column_log_accept(M, jtau, phi, s, s2, lg, beta)
            P[a, b] = math.exp(oracle.log_q(lg, s2)) * min(1.0, math.exp(la))
        P[a, a] = 1.0 - P[a].sum()
    E = np.array([oracle.column_energy(M, jtau, phi, c) for c in cols], float)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    assert np.abs(pi @ P - pi).max() < 1e-12
    # detailed balance, term by term
    F = pi[:, None] * P
    assert np.abs(F - F.T).max() < 1e-12
