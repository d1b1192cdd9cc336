"""Pins of the seeded input generators (``workloads.py``), CPU only.

The generators hold none of the method's arithmetic, but the batch and
serving size mixes, the record payloads and the explicit targets follow a
stated recipe.  They are checked here against an independent scalar
restatement built on the oracle's SplitMix64 (itself pinned to published
vectors in ``test_oracle.py``), against the closed-form moments of the
distributions they draw from, and for the structure the list and tree
generators promise.
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def test_uniforms_are_the_counter_based_splitmix_stream():
    # u_j = (mix(S ^ j) >> 11) * 2^-53, exactly, for the batch, size and
    # arrival streams
    for s in (5, 7, 11):
        u = workloads.uniforms(s, 300)
        for j in (0, 1, 2, 57, 299):
            assert u[j] == (oracle.splitmix64(s ^ j) >> 11) * 2.0 ** -53
        assert np.all((u >= 0.0) & (u < 1.0))


def test_log_uniform_sizes_follow_the_recipe():
    lo, hi, s = 8, 22, 7
    sizes = workloads.log_uniform_sizes(1000, lo, hi, s)
    u = workloads.uniforms(s, 1000)
    for j in range(0, 1000, 37):
        assert sizes[j] == min(max(math.floor(2.0 ** (lo + (hi - lo) * u[j])), 2 ** lo), 2 ** hi)
    assert sizes.min() >= 2 ** lo and sizes.max() <= 2 ** hi


def _log_uniform_moments(lo, hi):
    # X = 2^(lo + (hi - lo) U), U uniform on [0, 1): closed-form mean and sd
    d = (hi - lo) * math.log(2.0)
    m1 = (2.0 ** hi - 2.0 ** lo) / d
    m2 = (4.0 ** hi - 4.0 ** lo) / (2.0 * d)
    return m1, math.sqrt(m2 - m1 * m1)


def test_batch_workload_size_mix():
    sizes, seeds = workloads.batch_workload()
    assert sizes.shape == (8192,) and np.array_equal(seeds, np.arange(8192, dtype=np.uint64))
    mean, sd = _log_uniform_moments(8, 22)
    assert abs(sizes.mean() - mean) < 3 * sd / math.sqrt(8192)
    assert round(int(sizes.sum()) / 1e6) == 3504        # the 3.504e9 elements the batch bench moves
    # log-uniform: the exponents spread evenly over [8, 22)
    hist = np.histogram(np.log2(sizes), bins=14, range=(8, 22))[0]
    expected = 8192 / 14
    chi2 = float(((hist - expected) ** 2 / expected).sum())
    assert chi2 < 36.1                                  # chi-square, 13 df, p = 0.001


def test_serve_workload_mix():
    n = 20000
    sizes, dtypes, seeds, arrivals = workloads.serve_workload(count=n, rate_per_s=50.0)
    mean, sd = _log_uniform_moments(12, 28)
    assert abs(sizes.mean() - mean) < 3 * sd / math.sqrt(n)
    assert sizes.min() >= 2 ** 12 and sizes.max() <= 2 ** 28
    # dtype coin: low bit of mix(5 ^ j ^ 0xD1)
    for j in (0, 1, 2, 999, n - 1):
        want = "u64" if oracle.splitmix64(5 ^ j ^ 0xD1) & 1 else "u32"
        assert dtypes[j] == want
    frac = float(np.mean(dtypes == "u64"))
    assert abs(frac - 0.5) < 3 * math.sqrt(0.25 / n)
    assert np.array_equal(seeds, np.arange(n, dtype=np.uint64))
    # exponential inter-arrival gaps at the given rate: mean 1/rate, sd 1/rate
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert np.all(gaps >= 0.0)
    assert abs(gaps.mean() - 1 / 50.0) < 3 * (1 / 50.0) / math.sqrt(n)
    u = workloads.uniforms(11, 5)
    assert abs(gaps[3] - (-math.log1p(-u[3]) / 50.0)) < 1e-15


def test_record_payloads_are_splitmix_of_the_key():
    rec = workloads.records(1000)
    assert np.array_equal(rec[:, 0], np.arange(1000, dtype=np.uint64))
    for i in (0, 1, 2, 500, 999):
        assert int(rec[i, 1]) == oracle.splitmix64(i)


@pytest.mark.parametrize("n", [0, 1, 2, 1000, 100003])
def test_random_targets_are_in_range_and_uniform(n):
    H = workloads.random_targets(n, rng_seed=9)
    assert H.shape == (n,) and H.dtype == np.uint32
    i = np.arange(n)
    assert np.all(H <= i)
    if n >= 1000:
        # H[i] / (i + 1) is uniform on [0, 1): mean 1/2, sd 1/sqrt(12), up to
        # the flooring, which lowers the mean by 1/(2(i+1)) at most
        r = H[1:] / (i[1:] + 1.0)
        assert abs(r.mean() - 0.5) < 3 / math.sqrt(12 * (n - 1)) + np.mean(1 / (2 * (i[1:] + 1.0)))


@pytest.mark.parametrize("n,nlists", [(1, 1), (2, 1), (1000, 1), (1000, 7), (50000, 100)])
def test_random_lists_are_valid_lists(n, nlists):
    rec = workloads.random_lists(n, rng_seed=4, nlists=nlists)
    assert rec.shape == (n, 2) and rec.dtype == np.uint64
    assert oracle.list_check(rec) == 0
    heads = int(np.sum(rec[:, 0] == workloads.LIST_NIL))
    assert heads == min(nlists, n)


@pytest.mark.parametrize("leaves,trees", [(1, 1), (2, 1), (3, 1), (1000, 1), (1000, 9), (4097, 3)])
def test_random_trees_are_full_binary_forests(leaves, trees):
    rec = workloads.random_tree(leaves, rng_seed=6, trees=trees)
    n = rec.shape[0]
    t = min(trees, leaves)
    assert n == 2 * leaves - t                          # a full binary forest of t trees
    assert oracle.tree_check(rec) == 0
    nil = np.uint64(0xFFFFFFFFFFFFFFFF)
    assert int(np.sum(rec[:, 0] == nil)) == t           # one root per tree
    assert int(np.sum(rec[:, 1] == nil)) == leaves      # leaves have no children
