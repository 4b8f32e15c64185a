"""What the trained column proposal gains, measured on the 32x32 lattice x 32
slices system with 256 replicas (GPU).

The network is trained on 2^20 columns recorded from the plain sweep
(snapshots 10 sweeps apart after a 20000-sweep burn-in), then the plain chain
(sweep + PT per step) and the 1:1 chain (sweep + PT + learned pass) run from
the same state, with a second plain chain on other random numbers as a
control.  The test checks, and prints, that

* the trained network's proposals are accepted far more often than an
  untrained one's (the gain from training);
* on the fast-mixing temperatures the learned chain's energy and
  magnetisation histograms agree with the plain chain's within 3 standard
  errors as often as two chains of one law do: batch-mean standard errors
  (20 batches of 800 steps, tau_int below a hundredth of a batch),
  and a count of |z| > 3 bins no larger than the 0.999 quantile of its
  binomial law; a second plain chain continuing the same state on its own
  Philox seed passes the same bound and is not a replay of the first
  (its largest |z| is not 0) -- the Metropolis-Hastings correction keeps the
  Boltzmann law;
* at the coldest quarter of the ladder, where the single-spin sweep is nearly
  frozen, the learned chain reaches lower energies than the plain chain in
  the same number of steps.

A third chain interleaves the flip-symmetric mixture proposal (a second
network trained on the same snapshots in the orientation their spatial field
prefers); its histograms pass the same bound.

Reported, not asserted: the ESS/s ratios on the fast-mixing temperatures and
per inverse-temperature band (0.05-0.3, 0.3-1.0, 1.0-5.0; a temperature
counts where tau_int is below 1/50 of the run for both chains), and the
cold-end energy of a plain chain given the learned chain's device time (on
this system all favour the plain sweep: a learned pass costs about 0.9
sweeps, a mixture pass 1.4, and neither lowers tau_int per step by more
than ~15%).
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1004_0024_gb300 import ess, ising, workloads
    return ising, workloads, ess


def test_trained_proposal_gain(mods):
    ising, W, ess = mods
    # acceptance of an untrained network on an equilibrated state
    c = W.config1()
    sim = ising.Ising(c["graph"], c["betas"], seed=c["seed"], rng="philox", field_bits=16)
    sim.run(2000, 1)
    raw = ising.Mlp(32, seed=1)
    st = raw.learned_pass(sim)
    untrained = st["accepted"] / st["proposed"]
    raw.close()
    sim.close()

    out = ess.study(ising, W, burn=20000, n_steps=16000, epochs=6)
    out["untrained_accept_rate"] = untrained
    print(json.dumps(out, indent=1))
    assert out["accept_rate"] > 0.5 and out["accept_rate"] > 20 * untrained
    assert out["change_rate"] > 0.03
    assert out["loss_first_last"][1] < 0.8 * out["loss_first_last"][0]
    h, hc = out["histograms_learned_vs_plain"], out["histograms_plain_vs_plain"]
    assert out["fast_mixing_temps"] >= 20 and h["bins"] > 100
    assert hc["max_abs_z"] > 0.5, hc  # the control chain draws its own random numbers
    assert hc["beyond_3se"] <= hc["bound_beyond_3se"], hc
    assert h["beyond_3se"] <= h["bound_beyond_3se"], (h, hc)
    hm = out["mixture"]["histograms_vs_plain"]
    assert hm["bins"] > 100 and hm["beyond_3se"] <= hm["bound_beyond_3se"], (hm, hc)
    assert out["mixture_loss_first_last"][1] < 0.8 * out["mixture_loss_first_last"][0]
    assert len(out["bands_learned"]) == 3 and len(out["mixture"]["bands"]) == 3
    cq = out["coldest_quarter"]
    assert cq["mean_E_last_fifth_learned"] < cq["mean_E_last_fifth_plain"], cq
