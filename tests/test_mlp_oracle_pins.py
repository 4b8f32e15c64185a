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


def _ceil_p32_exact(bits):
    """ceil(p 2^32) of FP32 p in [0, 1] from the bit pattern, exact integer
    arithmetic: p = m 2^(e - 150) (m the 24-bit significand, e the biased
    exponent; e = 0 for subnormals with exponent 1 - 127 - 23)."""
    bits = bits.astype(np.uint64)
    e = (bits >> np.uint64(23)) & np.uint64(0xFF)
    m = (bits & np.uint64(0x7FFFFF)) | np.where(e > 0, np.uint64(0x800000), np.uint64(0))
    sh = np.where(e > 0, e.astype(np.int64), 1) - 150 + 32  # p 2^32 = m 2^sh
    out = np.zeros(bits.shape, dtype=np.uint64)
    pos = sh >= 0
    out[pos] = m[pos] << sh[pos].astype(np.uint64)
    neg = ~pos & (m > 0)
    k = (-sh[neg]).astype(np.uint64)
    big = k >= np.uint64(40)
    kk = np.minimum(k, np.uint64(39))
    out[neg] = np.where(big, np.uint64(1), (m[neg] + (np.uint64(1) << kk) - np.uint64(1)) >> kk)
    return out


def test_fp32_ceiling_of_proposal_thresholds_is_exact():
    """The learned-proposal kernel forms c = ceil(p 2^32) as ceilf(p * 2^32)
    in FP32 and decides u < c with a 32-bit compare (c = 2^32: always): for a
    strided sample of every FP32 p in [0, 1] (and the edge cases) this equals
    the integer ceiling, and u = c - 1 is below c while u = c is not."""
    one = np.float32(1.0).view(np.uint32)
    sample = np.arange(0, int(one) + 1, 97, dtype=np.uint32)
    edges = np.array([0, 1, 2, 0x007FFFFF, 0x00800000, 0x2F800000, 0x2F800001, 0x2F7FFFFF,
                      0x3F7FFFFF, int(one)], dtype=np.uint32)
    bits = np.unique(np.concatenate([sample, edges]))
    p = bits.view(np.float32)
    with np.errstate(over="ignore"):
        cf = np.ceil(p * np.float32(2.0 ** 32))  # FP32 throughout
    ci = _ceil_p32_exact(bits)
    assert np.array_equal(cf.astype(np.float64), ci.astype(np.float64))

    def word_below(u, c):  # the kernel's test u < c for an FP32 integer c <= 2^32
        full = c >= np.float32(2.0 ** 32)
        return full | (u < np.where(full, np.float32(0), c).astype(np.uint32))

    mid = (ci > 0) & (ci < np.uint64(1 << 32))
    c, cx = cf[mid], ci[mid]
    assert np.all(word_below((cx - np.uint64(1)).astype(np.uint32), c))   # u = c - 1: drawn +1
    assert not np.any(word_below(cx.astype(np.uint32), c))                # u = c: not drawn
    top = ci == np.uint64(1 << 32)                                        # p = 1: always +1
    assert top.any() and np.all(word_below(np.full(top.sum(), 0xFFFFFFFF, np.uint32), cf[top]))
    zero = ci == 0                                                        # p = 0: never
    assert zero.any() and not np.any(word_below(np.zeros(zero.sum(), np.uint32), cf[zero]))


def test_mixture_proposal_is_normalised_and_flip_symmetric():
    lg = np.array([0.3, -1.2, 2.0, 0.0, 4.5])
    cols = [np.array(c, np.int8) for c in itertools.product([-1, 1], repeat=lg.size)]
    tot = sum(math.exp(oracle.log_q_mix(lg, c)) for c in cols)
    assert abs(tot - 1.0) < 1e-12
    for c in cols:
        assert abs(oracle.log_q_mix(lg, c) - oracle.log_q_mix(lg, -c)) < 1e-12
        # half of q(c) plus half of q(-c), each from the independent law
        direct = 0.5 * math.exp(oracle.log_q(lg, c)) + 0.5 * math.exp(oracle.log_q(lg, -c))
        assert abs(math.exp(oracle.log_q_mix(lg, c)) - direct) < 1e-15


def test_mixture_of_uniform_proposal_is_uniform():
    lg = np.zeros(6)
    for c in itertools.product([-1, 1], repeat=6):
        assert abs(oracle.log_q_mix(lg, np.array(c, np.int8)) + 6 * math.log(2.0)) < 1e-12


def test_mixture_column_move_leaves_conditional_boltzmann_stationary():
    """Exact 2^M x 2^M matrix of one MH column move with the mixture of an
    arbitrary fixed proposal: exp(-beta E_col) is invariant and the flow is
    balanced term by term; a strongly one-sided q makes whole-column
    reversals likely proposals."""
    M, jtau, beta = 4, 3, 0.9
    phi = np.array([2, -1, 1, 3], np.int32)
    lg = np.array([2.4, 3.1, 1.7, 2.9])
    cols = [np.array(c, np.int8) for c in itertools.product([-1, 1], repeat=M)]
    n = len(cols)
    P = np.zeros((n, n))
    for a, s in enumerate(cols):
        for b, s2 in enumerate(cols):
            if a == b:
                continue
            la, dE = oracle.column_log_accept(M, jtau, phi, s, s2, lg, beta, mixture=True)
            assert dE == oracle.column_energy(M, jtau, phi, s2) - oracle.column_energy(M, jtau, phi, s)
            P[a, b] = math.exp(oracle.log_q_mix(lg, s2)) * min(1.0, math.exp(la))
        P[a, a] = 1.0 - P[a].sum()
    E = np.array([oracle.column_energy(M, jtau, phi, c) for c in cols], float)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    assert np.abs(pi @ P - pi).max() < 1e-12
    F = pi[:, None] * P
    assert np.abs(F - F.T).max() < 1e-12
    # all -1 (the reversal of the column q favours) is proposed a third of
    # the time: half of q(all +1) = prod_t sigma(l_t) = 0.70
    assert cols[0].tolist() == [-1] * M
    assert abs(math.exp(oracle.log_q_mix(lg, cols[0])) - 0.5 * math.exp(oracle.log_q(lg, -cols[0]))
               - 0.5 * math.exp(oracle.log_q(lg, cols[0]))) < 1e-15
    assert math.exp(oracle.log_q_mix(lg, cols[0])) > 0.35
