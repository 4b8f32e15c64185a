"""Effective sample size of Markov-chain time series, and the comparison of
the plain sweep with the sweep interleaved 1:1 with learned column passes.

``tau_int`` is Sokal's integrated autocorrelation time with his automatic
window (A. D. Sokal, "Monte Carlo Methods in Statistical Mechanics:
Foundations and New Algorithms", 1996): tau(W) = 1/2 + sum_{t=1..W} rho(t),
W the smallest window with W >= c tau(W), c = 5.  The effective sample size
of n correlated samples is n / (2 tau).

``compare`` drives the CUDA library only (no sampling on the host): it runs
both chains from the same state, records the energy and magnetisation of
every temperature index after each step, and times the steps separately
(CUDA events around steps enqueued back to back on the handle's stream).
"""
from __future__ import annotations

import time

import numpy as np


def autocorr(x: np.ndarray) -> np.ndarray:
    """Normalised autocorrelation rho(t), t = 0..n-1, by FFT (biased estimator)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    d = x - x.mean()
    var = d @ d / n
    if var == 0.0:
        out = np.zeros(n)
        out[0] = 1.0
        return out
    f = np.fft.rfft(d, 2 * n)
    acf = np.fft.irfft(f * np.conj(f))[:n] / n
    return acf / var


def tau_int(x: np.ndarray, c: float = 5.0) -> float:
    """Sokal's integrated autocorrelation time with the automatic window;
    0.5 for a constant series (no information beyond one sample)."""
    rho = autocorr(x)
    n = rho.size
    tau = 0.5
    for W in range(1, n):
        tau += rho[W]
        if W >= c * tau:
            return max(tau, 0.5)
    return max(tau, 0.5)


def ess(x: np.ndarray) -> float:
    x = np.asarray(x)
    return x.size / (2.0 * tau_int(x))


def mean_and_se(x: np.ndarray) -> tuple[float, float]:
    """Mean and its standard error sqrt(2 tau var / n)."""
    x = np.asarray(x, dtype=np.float64)
    return float(x.mean()), float(np.sqrt(2.0 * tau_int(x) * x.var() / x.size))


def histogram_agreement(a: np.ndarray, b: np.ndarray, bins: int = 8) -> np.ndarray:
    """z-scores of the bin fractions of two correlated series on shared edges
    (the standard error of each fraction from its indicator's tau)."""
    lo, hi = min(a.min(), b.min()), max(a.max(), b.max())
    if lo == hi:
        return np.zeros(0)
    edges = np.linspace(lo, hi + 1e-9 * max(1.0, abs(hi)), bins + 1)
    z = []
    for k in range(bins):
        ia = ((a >= edges[k]) & (a < edges[k + 1])).astype(np.float64)
        ib = ((b >= edges[k]) & (b < edges[k + 1])).astype(np.float64)
        ma, sa = mean_and_se(ia)
        mb, sb = mean_and_se(ib)
        s = np.hypot(sa, sb)
        if s > 0:
            z.append((ma - mb) / s)
    return np.asarray(z)


def _observe(sim, step, n_steps):
    """Run n_steps of ``step``, recording (E, m) per temperature after each."""
    Es, ms = [], []
    for _ in range(n_steps):
        step()
        E, m = sim.observables()
        Es.append(E)
        ms.append(m)
    return np.asarray(Es), np.asarray(ms)


def _seconds_per_step(sim, step, n_steps):
    """Device time per step of n_steps enqueued back to back (CUDA events on
    the handle's stream, no synchronisation in between)."""
    import torch

    stream = torch.cuda.current_stream()
    sim.set_stream(stream.cuda_stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n_steps):
        step()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3 / n_steps


def compare(sim, net, n_steps: int, swap_every: int = 1, warm: int = 20, n_time: int = 200):
    """Plain chain (one sweep + PT per step) against the 1:1 chain (one sweep
    + PT, then one learned pass per step), both from the handle's current
    state.  Returns per-temperature ESS/s of E and m for both chains, the
    z-scores of their histogram comparison and the learned acceptance rate."""
    blob = sim.save()

    def plain():
        sim.run(1, swap_every)

    def learned():
        sim.run(1, swap_every)
        net.learned_pass(sim, sync=False)

    out = {}
    for name, step in (("plain", plain), ("learned", learned)):
        sim.load(blob)
        for _ in range(warm):
            step()
        sps = _seconds_per_step(sim, step, n_time)
        sim.load(blob)
        t0 = time.perf_counter()
        E, m = _observe(sim, step, n_steps)
        wall = time.perf_counter() - t0
        secs = sps * n_steps
        R = E.shape[1]
        essE = np.array([ess(E[:, k]) for k in range(R)])
        essM = np.array([ess(m[:, k]) for k in range(R)])
        out[name] = dict(E=E, m=m, seconds=secs, seconds_per_step=sps, wall=wall, ess_E=essE, ess_m=essM,
                         ess_E_per_s=essE / secs, ess_m_per_s=essM / secs)
    # acceptance counts from a separate short run (the timed passes do not
    # synchronise to report them)
    acc = [0, 0, 0]
    for _ in range(min(50, n_steps)):
        sim.run(1, swap_every)
        st = net.learned_pass(sim)
        acc[0] += st["accepted"]
        acc[1] += st["proposed"]
        acc[2] += st["changed"]
    sim.load(blob)
    out["accept_rate"] = acc[0] / max(1, acc[1])
    out["change_rate"] = acc[2] / max(1, acc[1])
    R = out["plain"]["E"].shape[1]
    z = [histogram_agreement(out["plain"][o][:, k], out["learned"][o][:, k])
         for o in ("E", "m") for k in range(R)]
    out["hist_z"] = np.concatenate([v for v in z if v.size])
    return out
