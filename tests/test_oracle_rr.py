"""Oracle pins for RR sets (Definition 2) and Lemma 1 (I(S) = n Pr[S covers R])."""
import numpy as np
import pytest

import inputs
from helpers import (ancestors, exact_influence_ic, exact_influence_lt_wc, within_chernoff)

ALWAYS = 0xFFFFFFFF


def test_p1_is_reverse_reachability(orc):
    el = inputs.rmat(8, 900, seed=2)
    thr = np.full(el.m, ALWAYS, np.uint32)
    g = orc.Graph(el.n, el.src, el.dst, orc.W_EXPLICIT, thr)
    p = orc.Pool(g, orc.IC, seed=11).grow(300)
    for R in p.sets():
        Rs = set(int(x) for x in R)
        # with every edge live, R is {source} plus all its ancestors, for one source in R
        assert any(ancestors(el.n, el.src, el.dst, r) == Rs for r in Rs)


def test_p0_gives_singletons_with_uniform_sources(orc):
    n = 64
    el = inputs.rmat(6, 500, seed=2)
    g = orc.Graph(n, el.src, el.dst, orc.W_EXPLICIT, np.zeros(el.m, np.uint32))
    p = orc.Pool(g, orc.IC, seed=3).grow(64 * 400)
    off, nodes = p.arrays()
    assert np.all(np.diff(off) == 1)
    hist = np.bincount(nodes, minlength=n)
    exp = len(nodes) / n
    assert ((hist - exp) ** 2 / exp).sum() < 130  # 63 dof, p ~ 1e-6


def test_lt_path_returns_upstream(orc):
    # path 0 -> 1 -> ... -> 9: d_in = 1 everywhere on the path, w = 1
    L = 10
    el = inputs.edges(L, [(i, i + 1) for i in range(L - 1)])
    g = orc.Graph.from_edges(el, orc.W_WC)
    for R in orc.Pool(g, orc.LT, seed=5).grow(200).sets():
        top = int(R.max())
        assert list(R) == list(range(top + 1))
    for R in orc.Pool(g, orc.IC, seed=5).grow(200).sets():
        top = int(R.max())
        assert list(R) == list(range(top + 1))


def test_sets_sorted_unique(orc):
    el = inputs.rmat(11, 1 << 14, seed=8)
    g = orc.Graph.from_edges(el, orc.W_WC)
    for model in (orc.IC, orc.LT):
        for R in orc.Pool(g, model, seed=2).grow(500).sets():
            assert np.all(np.diff(R) > 0)


def _tiny_graphs():
    # <= 16 edges so that live-edge enumeration is exact
    yield inputs.edges(6, [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (4, 5), (5, 3), (2, 5), (1, 0)])
    yield inputs.edges(7, [(0, 1), (1, 2), (2, 0), (3, 0), (3, 4), (4, 5), (5, 6), (6, 4), (0, 6), (2, 5),
                           (1, 4), (6, 3)])


@pytest.mark.parametrize("gi", [0, 1])
@pytest.mark.parametrize("weighting", ["wc", "explicit"])
def test_ic_lemma1_exact_enumeration(orc, gi, weighting):
    el = list(_tiny_graphs())[gi]
    if weighting == "wc":
        g = orc.Graph.from_edges(el, orc.W_WC)
    else:
        rng = np.random.default_rng(gi)
        thr = (rng.uniform(0.05, 0.9, el.m) * 2**32).astype(np.uint32)
        g = orc.Graph.from_edges(el, orc.W_EXPLICIT, thr=thr)
    off, src, thr = g.csr()
    dst = np.repeat(np.arange(el.n), np.diff(off))
    N = 200_000
    p = orc.Pool(g, orc.IC, seed=17).grow(N)
    for S in ([0], [3], [1, 4], [2, 5, 6 % el.n]):
        I = exact_influence_ic(el.n, src, dst, thr, S)
        mu = I / el.n
        est = p.coverage(0, N, S) / N
        assert within_chernoff(est, mu, N), (S, I, est * el.n)


@pytest.mark.parametrize("gi", [0, 1])
def test_lt_lemma1_exact_enumeration(orc, gi):
    el = list(_tiny_graphs())[gi]
    g = orc.Graph.from_edges(el, orc.W_WC)
    N = 200_000
    p = orc.Pool(g, orc.LT, seed=23).grow(N)
    for S in ([0], [3], [1, 4]):
        I = exact_influence_lt_wc(el.n, el.src, el.dst, S)
        est = p.coverage(0, N, S) / N
        assert within_chernoff(est, I / el.n, N), (S, I, est * el.n)


def test_closed_form_star_and_path(orc):
    p_edge = 0.3
    t = np.uint32(int(p_edge * 2**32))
    pe = int(t) / 2**32
    # out-star c -> l_i: I({c}) = 1 + (n-1) p
    n = 12
    el = inputs.edges(n, [(0, i) for i in range(1, n)])
    g = orc.Graph.from_edges(el, orc.W_EXPLICIT, thr=np.full(el.m, t))
    N = 300_000
    pool = orc.Pool(g, orc.IC, seed=31).grow(N)
    I = 1 + (n - 1) * pe
    assert within_chernoff(pool.coverage(0, N, [0]) / N, I / n, N)
    # path v0 -> ... -> v_{L-1}: I({v0}) = sum_{i<L} p^i
    L = 8
    el = inputs.edges(L, [(i, i + 1) for i in range(L - 1)])
    g = orc.Graph.from_edges(el, orc.W_EXPLICIT, thr=np.full(el.m, t))
    pool = orc.Pool(g, orc.IC, seed=37).grow(N)
    I = sum(pe ** i for i in range(L))
    assert within_chernoff(pool.coverage(0, N, [0]) / N, I / L, N)


def test_wris_sources_follow_benefit(orc):
    n = 32
    el = inputs.edges(n, [(0, 1)])
    g = orc.Graph.from_edges(el, orc.W_EXPLICIT, thr=np.zeros(1, np.uint32))
    rng = np.random.default_rng(3)
    b = rng.integers(0, 50, n).astype(np.uint32)
    b[5] = 0
    b[6] = 1000
    N = 100_000
    pool = orc.Pool(g, orc.IC, seed=41, benefit=b).grow(N)
    _, nodes = pool.arrays()
    hist = np.bincount(nodes, minlength=n)
    assert hist[5] == 0 and np.all(hist[b == 0] == 0)
    exp = b / b.sum() * N
    nz = exp > 0
    chi2 = ((hist[nz] - exp[nz]) ** 2 / exp[nz]).sum()
    assert chi2 < 100


def test_keyed_independence_of_order(orc):
    # the same (seed, stream, j) gives the same set whether drawn in a pool or alone
    el = inputs.rmat(10, 1 << 13, seed=6)
    g = orc.Graph.from_edges(el, orc.W_WC)
    pool = orc.Pool(g, orc.IC, seed=99, stream=3).grow(50)
    sets = pool.sets()
    for j in (0, 7, 49):
        assert np.array_equal(orc.rr_set(g, orc.IC, 99, 3, j), sets[j])
    other = orc.Pool(g, orc.IC, seed=99, stream=4).grow(50).sets()
    assert any(not np.array_equal(a, b) for a, b in zip(sets, other))


@pytest.mark.parametrize("gi", [0, 1])
def test_lt_general_weights_lemma1(orc, gi):
    # LT with explicit in-weights summing to at most 1 (Sec. 2.1): exact enumeration vs RIS estimate
    from helpers import exact_influence_lt_general
    el = list(_tiny_graphs())[gi]
    rng = np.random.default_rng(40 + gi)
    d = np.bincount(el.dst, minlength=el.n)
    # random weights per in-edge scaled so each node's in-weights sum to a random value <= 1
    w = rng.uniform(0.2, 1.0, el.m)
    tot = np.zeros(el.n)
    np.add.at(tot, el.dst, w)
    scale = rng.uniform(0.5, 1.0, el.n) / np.maximum(tot, 1e-9)
    thr = np.floor(w * scale[el.dst] * 2**32).astype(np.uint64)
    thr = np.minimum(thr, 2**32 - 1).astype(np.uint32)
    g = orc.Graph.from_edges(el, orc.W_EXPLICIT, thr=thr)
    off, src, t2 = g.csr()
    dst = np.repeat(np.arange(el.n), np.diff(off))
    N = 200_000
    p = orc.Pool(g, orc.LT, seed=29).grow(N)
    for S in ([0], [3], [1, 4]):
        I = exact_influence_lt_general(el.n, src, dst, t2, S)
        est = p.coverage(0, N, S) / N
        assert within_chernoff(est, I / el.n, N), (S, I, est * el.n)
    assert d.sum() == el.m


@pytest.mark.parametrize("model", [0, 1])
def test_threaded_sampling_equals_one_thread(orc, model):
    # the all-cores CPU baseline splits sample ids into ranges over threads; every
    # RR set is a function of its key, so totals equal one thread's pool
    el = inputs.rmat(12, 1 << 15, seed=2)
    g = orc.Graph.from_edges(el, orc.W_WC)
    pool = orc.Pool(g, model, seed=9, stream=3).grow(1500)
    off, _ = pool.arrays()
    for threads in (1, 3, 8):
        used, entries, ev = orc.sample_threads(g, model, 9, 3, 0, 1500, threads)
        assert used == threads
        assert entries == off[-1] and ev == pool.edge_visits
    # a range that starts past 0
    used, entries, _ = orc.sample_threads(g, model, 9, 3, 500, 1000, 4)
    assert entries == off[1500] - off[500]
