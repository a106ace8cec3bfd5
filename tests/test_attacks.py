"""Attack-rate functions and injection samplers (paper table of time-exciting
attack strategies; App. "Sampling algorithm") against what their definitions
fix: closed-form values of g, the Poisson thinning law (counts and the
accepted-time distribution), the folded-normal candidate gaps of ND, the
piecewise weights of DRP, and the merge into a window."""
import numpy as np
import pytest
from scipy import stats

from paper_2411_10258_gb300.workload import attacks


def test_rate_closed_forms():
    t = np.array([0.25, 0.5, 0.9])
    np.testing.assert_allclose(attacks.rate("PLA", t, dict(a=2.0, b=3.0)), 2.0 * t ** 3)
    p = dict(W1=0.3, a1=2.0, W2=0.4, a2=1.5, gamma=3.0, t1=0.6)
    np.testing.assert_allclose(attacks.rate("DEA", t, p),
                               [0.3 * 2.0 * 0.25, 0.3 * 2.0 * 0.5, 0.4 * 1.5 * np.exp(3.0 * 0.3)])
    p = dict(C=2.0, gamma=10.0, t0=0.5)  # the denominator is 4 at t0
    np.testing.assert_allclose(attacks.rate("ASA", 0.5, p), 2.0 * np.exp(5.0) / 4.0)
    np.testing.assert_allclose(attacks.rate("DAM", t, dict(w=1.0, a1=3.0, a2=4.0)), 3.0 * t ** 2)
    np.testing.assert_allclose(attacks.rate("DAM", t, dict(w=0.0, a1=3.0, a2=4.0)), 4.0 * np.exp(4.0 * t))


def test_npp_constant_rate_is_poisson():
    rng = np.random.default_rng(1)
    counts, gaps = [], []
    for _ in range(200):
        s = attacks.sample("NPP", "PLA", rng, dict(a=1.0, b=0.0))  # g constant: every candidate kept
        counts.append(len(s))
        gaps.append(np.diff(np.concatenate([[0.0], s])))
    counts = np.asarray(counts)
    # Poisson(512) counts on [0, 1)
    assert abs(counts.mean() - 512) < 5 * np.sqrt(512 / len(counts))
    assert abs(counts.var() / 512 - 1.0) < 0.3
    assert stats.kstest(np.concatenate(gaps), "expon", args=(0, 1 / 512)).pvalue > 1e-3


def test_npp_thinning_follows_the_rate():
    rng = np.random.default_rng(2)
    ts = np.concatenate([attacks.sample("NPP", "PLA", rng, dict(a=3.0, b=1.0)) for _ in range(100)])
    # g(t) = 3t on [0, 1), g_max = 3: 256 kept per window on average, density 2t
    assert abs(len(ts) / 100 - 256) < 5 * np.sqrt(256 / 100)
    assert stats.kstest(ts, lambda x: np.clip(x, 0, 1) ** 2).pvalue > 1e-3


def test_nd_candidate_gaps_are_folded_normal():
    rng = np.random.default_rng(3)
    s = attacks.sample("ND", "PLA", rng, dict(a=1.0, b=0.0), lo=0.0, hi=20.0)
    gaps = np.diff(s)
    mu, sd = 1 / 512, 1 / 1024
    cdf = lambda x: stats.norm.cdf((x - mu) / sd) - stats.norm.cdf((-x - mu) / sd)
    assert stats.kstest(gaps, cdf).pvalue > 1e-3


def test_drp_weights_and_range():
    rng = np.random.default_rng(4)
    for _ in range(20):
        s = attacks.sample("DRP", "DAM", rng, lo=0.0, hi=1.0)
        assert len(s) > 0 and np.all((s >= 0) & (s < 1)) and np.all(np.diff(s) > 0)
    # the third with the smallest weight of the power-law part carries the exponential
    # burst: later thirds hold more of the kept times on average
    counts = np.zeros(3)
    for _ in range(200):
        s = attacks.sample("DRP", "DAM", rng)
        counts += np.bincount(np.minimum((s * 3).astype(int), 2), minlength=3)
    assert counts[2] > counts[1] > counts[0]


@pytest.mark.parametrize("strategy", attacks.STRATEGIES)
def test_every_strategy_samples(strategy):
    rng = np.random.default_rng(5)
    for sampler in ("NPP", "ND"):
        s = attacks.sample(sampler, strategy, rng)
        assert len(s) > 10 and np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < 1


def test_inject_merges_in_time_order():
    t = np.array([0.5, 1.0, 2.0, 3.0])
    ids = np.array([0, 1, 0, 2])
    tt, ii = attacks.inject(t, ids, 4.0, np.array([0.125, 0.5]), 3)
    np.testing.assert_array_equal(tt, [0.5, 0.5, 1.0, 2.0, 2.0, 3.0])
    np.testing.assert_array_equal(ii, [0, 3, 1, 0, 3, 2])
