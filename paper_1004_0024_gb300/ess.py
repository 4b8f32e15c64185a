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


N_BATCHES = 20  # batch means per series for the histogram standard errors


def batch_mean_and_se(x: np.ndarray, n_batches: int = N_BATCHES) -> tuple[float, float]:
    """Mean and its standard error from the spread of `n_batches` contiguous
    batch means (valid when a batch is much longer than tau_int; the first
    len(x) mod n_batches samples are dropped)."""
    x = np.asarray(x, dtype=np.float64)
    b = x.size // n_batches
    if b < 1:
        raise ValueError("fewer samples than batches")
    bm = x[x.size - b * n_batches:].reshape(n_batches, b).mean(axis=1)
    return float(bm.mean()), float(bm.std(ddof=1) / np.sqrt(n_batches))


def histogram_agreement(a: np.ndarray, b: np.ndarray, bins: int = 8,
                        n_batches: int = N_BATCHES) -> np.ndarray:
    """z-scores of the bin fractions of two correlated series.  The edges are
    quantiles of the pooled samples (so every bin holds a fair share of both
    series; tied values of an integer observable merge bins); the standard
    error of each fraction comes from batch means of its indicator series."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    pooled = np.concatenate([a, b])
    if pooled.min() == pooled.max():
        return np.zeros(0)
    inner = np.unique(np.quantile(pooled, np.arange(1, bins) / bins))
    edges = np.concatenate([[-np.inf], inner, [np.inf]])
    z = []
    for k in range(edges.size - 1):
        ia = ((a >= edges[k]) & (a < edges[k + 1])).astype(np.float64)
        ib = ((b >= edges[k]) & (b < edges[k + 1])).astype(np.float64)
        ma, sa = batch_mean_and_se(ia, n_batches)
        mb, sb = batch_mean_and_se(ib, n_batches)
        s = np.hypot(sa, sb)
        if s > 0:
            z.append((ma - mb) / s)
    return np.asarray(z)


def beyond_3se_law(bins: int, n_batches: int = N_BATCHES, q: float = 0.999) -> dict:
    """What two chains of the same law give: each z above is approximately
    Student-t with 2 (n_batches - 1) degrees of freedom (two batch-mean
    standard errors of similar size), so |z| > 3 has probability p; of
    `bins` such z-scores the count beyond 3 is about Binomial(bins, p)
    (bins of one histogram are not independent, which widens the law a
    little).  Returns p, the expected count and the q-quantile used as the
    bound of the check."""
    from scipy import stats
    p = float(2.0 * stats.t.sf(3.0, 2 * (n_batches - 1)))
    return {"p": p, "expected": p * bins, "bound": int(stats.binom.ppf(q, bins, p)), "quantile": q}


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


def compare(sim, net, n_steps: int, swap_every: int = 1, warm: int = 20, n_time: int = 200, ctrl=None,
            ctrl_seed: int | None = None, mix_net=None):
    """Plain chain (one sweep + PT per step) against the 1:1 chain (one sweep
    + PT, then one learned pass per step), both from the handle's current
    state.  With ``ctrl`` (a second handle of the same configuration, Philox
    streams) a second plain chain runs from the same state with other random
    numbers: after loading the shared state its seed is set to ``ctrl_seed``
    (the loaded checkpoint carries the first chain's key), so the spread
    between two correct chains calibrates the comparison.  With ``mix_net``
    a "mixture" chain interleaves learned passes of that network with the
    flip-symmetric mixture proposal.  Returns per-temperature series, ESS and
    ESS/s of E and m, and the learned acceptance and change rates."""
    blob = sim.save()
    if ctrl is not None and ctrl_seed is None:
        raise ValueError("a control chain needs its own seed")

    def plain():
        sim.run(1, swap_every)

    def learned():
        sim.run(1, swap_every)
        net.learned_pass(sim, sync=False)

    def plain_ctrl():
        ctrl.run(1, swap_every)

    def mixture():
        sim.run(1, swap_every)
        mix_net.learned_pass(sim, sync=False, mixture=True)

    chains = [("plain", sim, plain), ("learned", sim, learned)]
    if mix_net is not None:
        chains.append(("mixture", sim, mixture))
    if ctrl is not None:
        chains.append(("plain_ctrl", ctrl, plain_ctrl))
    out = {}

    def restart(name, h):
        h.load(blob)
        if name == "plain_ctrl":
            h.set_seed(ctrl_seed)

    for name, h, step in chains:
        restart(name, h)
        for _ in range(warm):
            step()
        sps = _seconds_per_step(h, step, n_time)
        restart(name, h)
        t0 = time.perf_counter()
        E, m = _observe(h, step, n_steps)
        wall = time.perf_counter() - t0
        secs = sps * n_steps
        R = E.shape[1]
        essE = np.array([ess(E[:, k]) for k in range(R)])
        essM = np.array([ess(m[:, k]) for k in range(R)])
        out[name] = dict(E=E, m=m, seconds=secs, seconds_per_step=sps, wall=wall, ess_E=essE, ess_m=essM,
                         ess_E_per_s=essE / secs, ess_m_per_s=essM / secs)
    # the plain chain for the device time the learned chain took: the same
    # number of observed steps at the end (the coldest temperatures barely
    # move under the plain sweep, so they are compared by the energy reached)
    tail = max(1, n_steps // 5)
    total = int(round(n_steps * out["learned"]["seconds_per_step"] / out["plain"]["seconds_per_step"]))
    sim.load(blob)
    if total > tail:
        sim.run(total - tail, swap_every)
    E, _ = _observe(sim, plain, tail)
    out["plain_equal_time"] = {"steps": max(total, tail), "E_tail": E}
    # acceptance counts from a separate short run (the timed passes do not
    # synchronise to report them)
    sim.load(blob)
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
    if mix_net is not None:
        acc = [0, 0, 0]
        for _ in range(min(50, n_steps)):
            sim.run(1, swap_every)
            st = mix_net.learned_pass(sim, mixture=True)
            acc[0] += st["accepted"]
            acc[1] += st["proposed"]
            acc[2] += st["changed"]
        sim.load(blob)
        out["mixture_accept_rate"] = acc[0] / max(1, acc[1])
        out["mixture_change_rate"] = acc[2] / max(1, acc[1])
    return out


BANDS = ((0.05, 0.3), (0.3, 1.0), (1.0, 5.0 + 1e-9))


def band_summary(res: dict, betas, chain: str, bands=BANDS, max_tau_frac: float = 1.0 / 50) -> list:
    """ESS/s of ``chain`` against the plain chain per inverse-temperature band:
    per temperature of the band, E and m count where both chains pass the
    split-half check and have tau_int below max_tau_frac of the run (so that
    tau is estimated from at least 50 autocorrelation times); the band reports
    how many temperatures qualified, the median ESS/s ratio over them and
    the median tau_int of each chain."""
    P, L = res["plain"], res[chain]
    n = P["E"].shape[0]
    betas = np.asarray(betas)
    out = []
    for lo, hi in bands:
        ks = np.nonzero((betas >= lo) & (betas < hi))[0]
        row = {"betas": [float(lo), float(min(hi, betas.max()))], "temps": int(ks.size)}
        for o in ("E", "m"):
            good, ratio, tp, tl = [], [], [], []
            for k in ks:
                xp, xl = P[o][:, k], L[o][:, k]
                if not (equilibrated(xp) and equilibrated(xl)):
                    continue
                a, b = tau_int(xp), tau_int(xl)
                if max(a, b) >= max_tau_frac * n:
                    continue
                good.append(int(k))
                ratio.append(L[f"ess_{o}_per_s"][k] / P[f"ess_{o}_per_s"][k])
                tp.append(a)
                tl.append(b)
            row[o] = {"qualified": len(good),
                      "ess_per_s_ratio_median": float(np.median(ratio)) if ratio else None,
                      "ess_per_s_ratio_min_max": [float(np.min(ratio)), float(np.max(ratio))] if ratio else None,
                      "tau_int_median_plain": float(np.median(tp)) if tp else None,
                      f"tau_int_median_{chain}": float(np.median(tl)) if tl else None}
        out.append(row)
    return out


def equilibrated(x: np.ndarray) -> bool:
    """Both halves of the series have means within 3 standard errors and the
    series is not constant."""
    x = np.asarray(x, dtype=np.float64)
    if x.min() == x.max():
        return False
    h = x.size // 2
    m1, s1 = mean_and_se(x[:h])
    m2, s2 = mean_and_se(x[h:])
    return abs(m1 - m2) < 3.0 * max(np.hypot(s1, s2), 1e-300)


def fast_mixing(res: dict, names, max_tau_frac: float = 1.0 / (100 * N_BATCHES)) -> np.ndarray:
    """Temperatures where E and m of every named chain pass the split-half
    check with tau_int below max_tau_frac of the run (by default a hundredth
    of one batch of the histogram standard errors)."""
    R = res["plain"]["E"].shape[1]
    n = res["plain"]["E"].shape[0]
    ok = np.ones(R, dtype=bool)
    for name in names:
        for o in ("E", "m"):
            x = res[name][o]
            for k in range(R):
                if ok[k]:
                    ok[k] = equilibrated(x[:, k]) and tau_int(x[:, k]) < max_tau_frac * n
    return ok


def _hist_stats(res, a, b, temps):
    z = [histogram_agreement(res[a][o][:, k], res[b][o][:, k]) for o in ("E", "m") for k in np.nonzero(temps)[0]]
    z = np.concatenate(z) if z else np.zeros(0)
    law = beyond_3se_law(int(z.size)) if z.size else None
    return {"bins": int(z.size), "beyond_3se": int((np.abs(z) > 3).sum()),
            "max_abs_z": float(np.abs(z).max()) if z.size else None,
            "z_rms": float(np.sqrt(np.mean(z * z))) if z.size else None,
            "se": f"batch means ({N_BATCHES} batches per series), pooled-quantile bins",
            "expected_beyond_3se": law["expected"] if law else None,
            "bound_beyond_3se": law["bound"] if law else None}


def summarize(res: dict, betas) -> dict:
    """JSON-ready summary of ``compare``.  ESS/s ratios (learned / plain) are
    medians over the fast-mixing temperatures (split-half check passed, tau
    below a hundredth of a batch, for every chain); the histogram comparison is
    made there too, for learned vs plain and, as calibration, for the second
    plain chain vs plain.  The coldest quarter, where the plain sweep barely
    moves on this time scale, is reported by the energies reached."""
    P, L = res["plain"], res["learned"]
    R = P["E"].shape[1]
    names = ["plain", "learned"] + [k for k in ("plain_ctrl", "mixture") if k in res]
    fm = fast_mixing(res, names)
    out = {"accept_rate": res["accept_rate"], "change_rate": res["change_rate"],
           "ms_per_step": {"plain": 1e3 * P["seconds_per_step"], "learned": 1e3 * L["seconds_per_step"]},
           "steps": int(P["E"].shape[0]), "fast_mixing_temps": int(fm.sum()),
           "fast_mixing_betas": [float(betas[k]) for k in np.nonzero(fm)[0][[0, -1]]] if fm.any() else None}
    for o in ("E", "m"):
        ratio = L[f"ess_{o}_per_s"] / P[f"ess_{o}_per_s"]
        per_step = L[f"ess_{o}"] / P[f"ess_{o}"]
        out[o] = {"ess_per_s_ratio_median": float(np.median(ratio[fm])) if fm.any() else None,
                  "ess_per_step_ratio_median": float(np.median(per_step[fm])) if fm.any() else None,
                  "ess_per_s_plain_median": float(np.median(P[f"ess_{o}_per_s"][fm])) if fm.any() else None,
                  "ess_per_s_learned_median": float(np.median(L[f"ess_{o}_per_s"][fm])) if fm.any() else None}
    out["histograms_learned_vs_plain"] = _hist_stats(res, "learned", "plain", fm)
    out["bands_learned"] = band_summary(res, betas, "learned")
    if "mixture" in res:
        X = res["mixture"]
        out["mixture"] = {"accept_rate": res.get("mixture_accept_rate"), "change_rate": res.get("mixture_change_rate"),
                          "ms_per_step": 1e3 * X["seconds_per_step"],
                          "histograms_vs_plain": _hist_stats(res, "mixture", "plain", fm),
                          "bands": band_summary(res, betas, "mixture")}
        for o in ("E", "m"):
            ratio = X[f"ess_{o}_per_s"] / P[f"ess_{o}_per_s"]
            out["mixture"][o] = {"ess_per_s_ratio_median": float(np.median(ratio[fm])) if fm.any() else None}
    if "plain_ctrl" in res:
        out["histograms_plain_vs_plain"] = _hist_stats(res, "plain_ctrl", "plain", fm)
    cold = slice(3 * R // 4, R)
    eP, eL = P["E"][:, cold], L["E"][:, cold]
    tail = max(1, eP.shape[0] // 5)
    out["coldest_quarter"] = {"betas": [float(betas[3 * R // 4]), float(betas[R - 1])],
                              "mean_E_last_fifth_plain": float(eP[-tail:].mean()),
                              "mean_E_last_fifth_learned": float(eL[-tail:].mean()),
                              "min_E_plain": int(eP.min()), "min_E_learned": int(eL.min())}
    if "plain_equal_time" in res:
        et = res["plain_equal_time"]
        out["coldest_quarter"]["plain_equal_time_steps"] = et["steps"]
        out["coldest_quarter"]["mean_E_last_fifth_plain_equal_time"] = float(et["E_tail"][:, cold].mean())
    return out


def study(ising, W, burn: int, n_steps: int, epochs: int, records: int = 1 << 20, seed_net: int = 1):
    """The learned-proposal study on the 32x32x32 system (Philox streams, so
    that a control handle can continue the same state with other random
    numbers): burn-in, record `records` columns (snapshots 10 sweeps apart),
    train, compare."""
    c = W.config1()
    sim = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng="philox", field_bits=c["field_bits"])
    ctrl = ising.Ising(c["graph"], c["betas"], seed=c["seed"] + 7919, rng="philox", field_bits=c["field_bits"])
    done = 0
    while done < burn:
        k = min(1000, burn - done)
        sim.run(k, 1)
        done += k
    S = c["graph"].n // c["graph"].n_slices
    # two networks on the same snapshots: the independent proposal on the
    # columns as sampled, the mixture proposal on the columns in the
    # orientation their spatial field prefers
    net = ising.Mlp(c["graph"].n_slices, seed=seed_net, capacity=records)
    mix = ising.Mlp(c["graph"].n_slices, seed=seed_net + 1, capacity=records)
    while net.n_records + c["R"] * S <= records:
        sim.run(10, 1)
        net.collect(sim)
        mix.collect(sim, oriented=True)
    t0 = time.perf_counter()
    losses = [net.train(1, 4096, 1e-3) for _ in range(epochs)]
    losses_mix = [mix.train(1, 4096, 1e-3) for _ in range(epochs)]
    train_s = time.perf_counter() - t0
    res = compare(sim, net, n_steps, ctrl=ctrl, ctrl_seed=c["seed"] + 7919, mix_net=mix)
    out = summarize(res, c["betas"])
    # the fused network kernel alone, timed with CUDA events around each launch
    net.set_profiling(True)
    for _ in range(20):
        net.learned_pass(sim, sync=False)
    prof = net.stats()
    net.set_profiling(False)
    M = c["graph"].n_slices
    flop = 2 * ((M + 1) * 256 + 256 * 256 + 256 * M)  # per column, 33 -> 256 -> 256 -> 32
    out["network"] = {"launches": prof["network_launches"], "columns": prof["network_rows"],
                      "ms": prof["network_ms"], "flop_per_column": flop,
                      "tflops": prof["network_rows"] * flop / (prof["network_ms"] * 1e-3) / 1e12
                      if prof["network_ms"] > 0 else None}
    out.update({"burn_in_sweeps": burn, "records": int(net.n_records), "epochs": epochs,
                "loss_first_last": [losses[0], losses[-1]] if losses else None,
                "mixture_loss_first_last": [losses_mix[0], losses_mix[-1]] if losses_mix else None,
                "train_seconds": train_s, "rng": "philox"})
    mix.close()
    net.close()
    ctrl.close()
    sim.close()
    return out
