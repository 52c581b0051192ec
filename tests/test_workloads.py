"""Seeded input generators (host side): the Zipf(s = 1) query order.

The benchmark's second query batch draws keys in a Zipf order with exponent 1:
rank r of n with probability (1/r) / H_n.  The sampler must give exactly that
law, not a continuous approximation of it.
"""
import numpy as np
import pytest
from scipy import stats

from paper_2404_18497_b300 import workloads


def _chi2(counts: np.ndarray, n: int) -> float:
    p = 1.0 / np.arange(1, n + 1)
    e = p / p.sum() * counts.sum()
    return float(((counts - e) ** 2 / e).sum())


@pytest.mark.parametrize("n", [2, 3, 10, 57, 400])
def test_zipf_rank_frequencies_are_one_over_r_h_n(n):
    rng = np.random.default_rng(n)
    q = 2_000_000
    r = workloads.zipf_ranks(n, q, rng)
    assert r.min() >= 1 and r.max() <= n
    c = np.bincount(r, minlength=n + 1)[1:]
    assert _chi2(c, n) < stats.chi2.ppf(1 - 1e-6, n - 1), n
    # the most frequent rank within 5 standard deviations of q / H_n
    h = (1.0 / np.arange(1, n + 1)).sum()
    assert abs(c[0] - q / h) < 5 * np.sqrt(q / h)


def test_zipf_test_rejects_the_continuous_approximation():
    """The frequency test has the power to tell the exact law from floor((n+1)^u),
    the continuous inversion used before: at n = 10 that gives rank 1 with
    probability ln 2 / ln 11 = 0.289 instead of 1 / H_10 = 0.341."""
    n, q = 10, 2_000_000
    rng = np.random.default_rng(5)
    r = np.clip(np.floor(np.exp(rng.random(q) * np.log(n + 1.0))).astype(np.int64), 1, n)
    c = np.bincount(r, minlength=n + 1)[1:]
    assert _chi2(c, n) > stats.chi2.ppf(1 - 1e-6, n - 1)


def test_zipf_queries_are_members_and_seeded():
    keys = workloads.distinct_u64(5000, 3)
    a = workloads.zipf_queries(keys, 20_000, 9)
    b = workloads.zipf_queries(keys, 20_000, 9)
    assert np.array_equal(a, b) and np.isin(a, keys).all()
    assert workloads.zipf_ranks(1, 100, np.random.default_rng(0)).tolist() == [1] * 100
