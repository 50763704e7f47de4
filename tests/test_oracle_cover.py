"""Oracle pins for Cov (Eq. 1), Max-Coverage (Algorithm 2) and Estimate-Inf (Algorithm 3)."""
import math

import numpy as np
import pytest

import inputs
from helpers import brute_opt_coverage, coverage, exhaustive_greedy


def _random_system(rng, n, N):
    sets = []
    for _ in range(N):
        size = int(rng.integers(1, 5))
        sets.append(np.sort(rng.choice(n, size=size, replace=False)).astype(np.int32))
    return sets


@pytest.mark.parametrize("trial", range(12))
def test_greedy_matches_exhaustive_and_bound(orc, trial):
    rng = np.random.default_rng(100 + trial)
    n = int(rng.integers(5, 11))
    sets = _random_system(rng, n, int(rng.integers(3, 25)))
    k = int(rng.integers(1, min(4, n) + 1))
    seeds, gains, cov = orc.max_coverage_sets(n, sets, k)
    S_ref, cov_ref = exhaustive_greedy(n, sets, k)
    assert list(seeds) == S_ref          # same picks, smallest-id tie-break
    assert cov == cov_ref == coverage(sets, seeds) == int(gains.sum())
    assert np.all(np.diff(gains) <= 0)   # submodular: gains never increase
    opt = brute_opt_coverage(n, sets, k)
    assert cov >= (1 - 1 / math.e) * opt  # Nemhauser bound quoted in Sec. 4.1
    assert len(set(seeds.tolist())) == k


def test_greedy_zero_gain_picks_are_smallest_unused(orc):
    sets = [np.array([3], np.int32), np.array([3], np.int32)]
    seeds, gains, cov = orc.max_coverage_sets(6, sets, 4)
    assert list(seeds) == [3, 0, 1, 2] and list(gains) == [2, 0, 0, 0] and cov == 2


def test_pool_coverage_matches_bruteforce(orc):
    el = inputs.rmat(9, 1 << 12, seed=12)
    g = orc.Graph.from_edges(el, orc.W_WC)
    pool = orc.Pool(g, orc.IC, seed=4).grow(400)
    sets = pool.sets()
    rng = np.random.default_rng(1)
    for _ in range(5):
        S = rng.choice(el.n, 5, replace=False).astype(np.int32)
        assert pool.coverage(100, 400, S) == coverage(sets[100:400], S)
    cnt = pool.counts(400)
    ref = np.zeros(el.n, np.int64)
    for R in sets:
        ref[R] += 1
    assert np.array_equal(cnt, ref)
    seeds, gains, cov = pool.max_coverage(400, 8)
    assert cov == coverage(sets, seeds)


def test_estimate_inf_full_cover_closed_form(orc):
    # S = V covers every RR set: the stopping rule ends at T = ceil(Lambda2)
    el = inputs.rmat(8, 1000, seed=1)
    g = orc.Graph.from_edges(el, orc.W_WC)
    lam2 = 123.4
    T, hits, _ = orc.estimate_inf(g, orc.IC, 5, 2, np.arange(el.n), lam2, 10_000)
    assert T == 124 and hits == 124
    # T_max too small: the paper's -1 (here 0)
    T, hits, _ = orc.estimate_inf(g, orc.IC, 5, 2, np.arange(el.n), lam2, 100)
    assert T == 0 and hits == 100


def test_estimate_inf_lemma3_bound(orc):
    # S = {isolated node}: I(S) = 1, so successes ~ Bernoulli(1/n); Lemma 3 bounds
    # the estimate n*Lambda2/T above by (1+eps') I(S) w.p. >= 1 - delta'.
    n = 50
    el = inputs.edges(n, [(0, 1), (1, 2)])
    g = orc.Graph.from_edges(el, orc.W_WC)
    eps, delta = 0.2, 1e-3
    lam2 = 1 + (1 + eps) * orc.upsilon(eps, math.log(1 / delta))
    for seed in range(4):
        T, hits, _ = orc.estimate_inf(g, orc.IC, seed, 1, [40], lam2, 10**7)
        assert T > 0 and hits == math.ceil(lam2)
        est = n * lam2 / T
        assert est <= (1 + eps) * 1.0
        assert est >= (1 - 2 * eps) * 1.0  # lower side (not part of the lemma), loose
