"""The effective-sample-size estimator against processes with a known
integrated autocorrelation time (CPU)."""
import numpy as np
import pytest

from paper_1004_0024_gb300 import ess


@pytest.mark.parametrize("phi", [0.0, 0.5, 0.9, 0.97])
def test_tau_int_of_ar1(phi):
    # x_t = phi x_{t-1} + e_t has rho(t) = phi^t, tau_int = (1 + phi) / (2 (1 - phi))
    rng = np.random.default_rng(int(phi * 100))
    n = 400_000
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    exact = (1 + phi) / (2 * (1 - phi))
    assert abs(ess.tau_int(x) - exact) <= 0.05 * exact + 0.02


def test_autocorr_of_alternating_series():
    x = np.tile([1.0, -1.0], 500)
    rho = ess.autocorr(x)
    assert rho[0] == pytest.approx(1.0)
    assert rho[1] == pytest.approx(-(999 / 1000), abs=1e-12)


def test_constant_series_counts_as_one_sample_per_two():
    assert ess.tau_int(np.ones(100)) == 0.5


def test_mean_and_se_matches_batch_means():
    rng = np.random.default_rng(3)
    phi, n = 0.8, 200_000
    x = np.empty(n)
    x[0] = 0.0
    e = rng.normal(size=n)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    m, se = ess.mean_and_se(x)
    batches = x.reshape(200, -1).mean(axis=1)
    assert se == pytest.approx(batches.std(ddof=1) / np.sqrt(200), rel=0.25)


def test_histogram_agreement_flags_a_shift():
    rng = np.random.default_rng(4)
    a = rng.normal(size=20000)
    assert np.all(np.abs(ess.histogram_agreement(a, rng.normal(size=20000))) < 4)
    assert np.abs(ess.histogram_agreement(a, rng.normal(0.2, 1, size=20000))).max() > 6


def _ar1(rng, phi, n):
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi * phi)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x


def test_histogram_z_scores_of_two_chains_of_one_law_follow_their_stated_law():
    # pairs of independent AR(1) chains (tau_int = 4.5) of the run length used
    # by the learned-proposal study: the batch-mean z-scores must have unit
    # spread and a |z| > 3 count within the bound of beyond_3se_law
    rng = np.random.default_rng(11)
    z = np.concatenate([ess.histogram_agreement(_ar1(rng, 0.8, 4000), _ar1(rng, 0.8, 4000))
                        for _ in range(150)])
    law = ess.beyond_3se_law(z.size)
    assert z.size >= 150 * 7
    assert 0.85 < np.sqrt(np.mean(z * z)) < 1.15
    assert int((np.abs(z) > 3).sum()) <= law["bound"]
    assert 0.001 < law["p"] < 0.01


def test_histogram_agreement_detects_a_shifted_correlated_chain():
    rng = np.random.default_rng(12)
    z = np.concatenate([ess.histogram_agreement(_ar1(rng, 0.8, 4000), _ar1(rng, 0.8, 4000) + 0.5)
                        for _ in range(20)])
    assert int((np.abs(z) > 3).sum()) > ess.beyond_3se_law(z.size)["bound"]


def test_batch_mean_se_of_iid_samples():
    rng = np.random.default_rng(13)
    ses = [ess.batch_mean_and_se(rng.normal(size=4000))[1] for _ in range(400)]
    assert np.mean(ses) == pytest.approx(1 / np.sqrt(4000), rel=0.05)
