"""The seeded input generator that both sides consume: R-MAT edge lists are
unique, loop-free, sorted by (dst, src), and identical for any host thread
count (the container and the GPU machine have different core counts); the Zipf
benefit table is a keyed permutation of max(1, floor(2^20 / rank^s)); the
uniform doubles lie in [0, 1)."""
import numpy as np

import inputs


def test_rmat_unique_sorted_loop_free():
    el = inputs.rmat(10, 1 << 14, seed=3)
    assert el.n == 1024 and el.m > 0
    assert el.src.min() >= 0 and el.src.max() < el.n and el.dst.min() >= 0 and el.dst.max() < el.n
    assert not np.any(el.src == el.dst)
    key = el.dst.astype(np.int64) * el.n + el.src
    assert np.all(np.diff(key) > 0)  # strictly increasing: sorted and no duplicates


def test_rmat_independent_of_thread_count_and_keyed_by_seed():
    ref = inputs.rmat(12, 50_000, seed=9, threads=1)
    for t in (2, 3, 7, 16):
        el = inputs.rmat(12, 50_000, seed=9, threads=t)
        assert np.array_equal(el.src, ref.src) and np.array_equal(el.dst, ref.dst)
    other = inputs.rmat(12, 50_000, seed=10, threads=4)
    assert not (other.m == ref.m and np.array_equal(other.src, ref.src))


def test_rmat_skew_follows_the_quadrant_weights():
    # a = 0.57 on the (low, low) quadrant against d = 0.05 on (high, high)
    el = inputs.rmat(12, 1 << 16, seed=2)
    half = el.n // 2
    ll = np.sum((el.src < half) & (el.dst < half))
    hh = np.sum((el.src >= half) & (el.dst >= half))
    assert ll > 4 * hh


def test_zipf_benefit_is_a_keyed_permutation_of_the_rank_weights():
    n, s = 5000, 1.2
    w = inputs.zipf_benefit(n, s, seed=4)
    ranks = np.arange(1, n + 1, dtype=np.float64)
    want = np.maximum(1, np.floor(1048576.0 / ranks ** s)).astype(np.uint32)
    assert np.array_equal(np.sort(w), np.sort(want))
    assert np.array_equal(inputs.zipf_benefit(n, s, seed=4), w)
    assert not np.array_equal(inputs.zipf_benefit(n, s, seed=5), w)


def test_uniforms_in_unit_interval():
    u = inputs.uniforms(100_000, seed=7)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(inputs.uniforms(100_000, seed=7), u)
