"""Pins of the oracle's weighted-cascade gap form (IC, Sec. 2.1, with the
weights of Sec. 6.1).

Under IC each in-edge (u, v) is live on its own coin with probability
w(u, v); with weighted-cascade weights every in-edge of v has the same
probability p = t / 2^32, t = floor(2^32 / d_in(v)).  The oracle therefore draws
the runs of dead edges between live ones from the geometric law
P(G >= g) = q^g, q = 1 - p, in Q64 integer arithmetic.  These tests hold that
arithmetic to the mathematics, not to itself:

* the gap function against exact powers q^g (mpmath at 200 bits) at its
  thresholds, over in-degrees from 2 to 2^31 - 1;
* whole in-lists against the law of d independent coins: on a star whose
  centre is always the source, the number of live in-edges follows
  Binomial(d, p) exactly and every edge is equally likely to be live;
* whole RR sets on an R-MAT graph against the oracle's per-edge-coin path fed
  the same thresholds.
"""
import math

import numpy as np
import pytest

import inputs

mpmath = pytest.importorskip("mpmath")


def _q(d):
    t = (1 << 32) // d
    return mpmath.mpf((1 << 32) - t) / mpmath.mpf(1 << 32)


@pytest.mark.parametrize("d", [2, 3, 5, 7, 10, 64, 100, 1000, 4097, 65536, 1_000_003, (1 << 31) - 1])
def test_gap_thresholds_are_exact_powers(orc, d):
    """G(U) >= g exactly when U < q^g * 2^64, up to a relative d * 2^-59 at
    the threshold (the truncation of the squarings); checked just inside and
    just outside each threshold."""
    mpmath.mp.prec = 200
    q = _q(d)
    J = d.bit_length()
    rng = np.random.default_rng(d)
    gs = {1, 2, 3, d // 3, d // 2, d - 1, d, d + 1, (1 << J) - 1}
    gs |= {int(x) for x in rng.integers(1, 1 << J, size=24)}
    gs = sorted(g for g in gs if 1 <= g <= (1 << J) - 1)
    rel = max(2.0 ** -50, d * 2.0 ** -59)
    two64 = mpmath.mpf(2) ** 64
    for g in gs:
        X = q ** g * two64
        lo = int(mpmath.floor(X * (1 - rel))) - 1
        hi = int(mpmath.ceil(X * (1 + rel))) + 1
        if lo >= 0:
            assert orc.wc_gap(d, lo) >= g, (d, g)
        if hi < (1 << 64):
            assert orc.wc_gap(d, hi) < g, (d, g)
    # U at or above q: no dead edge before the next live one
    assert orc.wc_gap(d, (1 << 64) - 1) == 0
    # U = 0 is below every power: the largest gap, 2^J - 1 >= d (past the list)
    assert orc.wc_gap(d, 0) == (1 << J) - 1 >= d


def test_gap_small_cases_by_hand(orc):
    # d = 2: p = q = 1/2 exactly, J = 2; thresholds 2^63 (g=1), 2^62 (g=2), 2^61 (g=3)
    assert orc.wc_gap(2, (1 << 63) - 1) == 1 and orc.wc_gap(2, 1 << 63) == 0
    assert orc.wc_gap(2, (1 << 62) - 1) == 2 and orc.wc_gap(2, 1 << 62) == 1
    assert orc.wc_gap(2, (1 << 61) - 1) == 3 and orc.wc_gap(2, 1 << 61) == 2
    # d = 4: p = 1/4, q = 3/4: thresholds (3/4)^g 2^64, exact in Q64 for g <= 3 (J = 3)
    for g in range(1, 4):
        X = (3 ** g) << (64 - 2 * g)
        assert orc.wc_gap(4, X - 1) >= g and orc.wc_gap(4, X) == g - 1


def _star(d):
    # centre 0 with in-edges from 1..d; the leaves have none
    src = np.arange(1, d + 1, dtype=np.int32)
    dst = np.zeros(d, dtype=np.int32)
    return inputs.EdgeList(d + 1, src, dst)


@pytest.mark.parametrize("d", [1, 2, 3, 10, 1000])
def test_star_live_count_is_binomial(orc, d):
    from scipy.stats import binom, chi2

    el = _star(d)
    g = orc.Graph.from_edges(el, orc.W_WC)
    benefit = np.zeros(el.n, dtype=np.int64)
    benefit[0] = 1  # the centre is every set's source
    N = 20000
    pool = orc.Pool(g, orc.IC, seed=11, benefit=benefit).grow(N)
    sets = pool.sets()
    assert all(s[0] == 0 for s in sets)
    K = np.array([len(s) - 1 for s in sets])
    if d == 1:
        assert (K == 1).all()  # weight 1/1: the edge is always live
        return
    p = ((1 << 32) // d) / float(1 << 32)
    pmf = binom.pmf(np.arange(d + 1), d, p)
    # pool the tail so every cell expects at least 20 sets
    exp, obs = [], []
    acc_e, acc_o = 0.0, 0
    hist = np.bincount(K, minlength=d + 1)
    for k in range(d + 1):
        acc_e += N * pmf[k]
        acc_o += hist[k]
        if acc_e >= 20 and N * pmf[k + 1:].sum() >= 20:
            exp.append(acc_e)
            obs.append(acc_o)
            acc_e, acc_o = 0.0, 0
    exp.append(acc_e)
    obs.append(acc_o)
    exp, obs = np.array(exp), np.array(obs)
    stat = ((obs - exp) ** 2 / exp).sum()
    assert stat < chi2.ppf(1 - 1e-4, len(exp) - 1), (stat, obs, exp)
    # every in-edge equally likely: inclusion counts of the leaves
    inc = np.bincount(np.concatenate([s[1:] for s in sets]), minlength=d + 1)[1:]
    e = N * p
    stat2 = ((inc - e) ** 2 / e).sum()
    assert stat2 < chi2.ppf(1 - 1e-4, d - 1), stat2


def test_star_mean_matches_coins_at_a_hub(orc):
    # d = 100000: E[K] = d t / 2^32 (just under 1), Var = d p q; 4000 sets
    d = 100_000
    el = _star(d)
    g = orc.Graph.from_edges(el, orc.W_WC)
    benefit = np.zeros(el.n, dtype=np.int64)
    benefit[0] = 1
    N = 4000
    sets = orc.Pool(g, orc.IC, seed=3, benefit=benefit).grow(N).sets()
    K = np.array([len(s) - 1 for s in sets], dtype=np.float64)
    p = ((1 << 32) // d) / float(1 << 32)
    mean, sd = d * p, math.sqrt(d * p * (1 - p) / N)
    assert abs(K.mean() - mean) < 5 * sd
    # P(K = 0) = q^d
    p0 = (1 - p) ** d
    assert abs((K == 0).mean() - p0) < 5 * math.sqrt(p0 * (1 - p0) / N)


def test_gap_form_matches_coins_on_rmat(orc):
    """Whole RR sets: the weighted-cascade gap form against independent per-edge
    coins of the same probabilities (the explicit-threshold path with
    t = floor(2^32 / d_in), which draws one coin per in-edge), on an R-MAT
    graph: same distribution of set sizes (two-sample KS), same mean size and
    the same coverage of the most covered nodes."""
    from scipy.stats import ks_2samp

    el = inputs.rmat(14, 1 << 17, seed=1)
    d_in = np.bincount(el.dst, minlength=el.n)
    thr = np.where(d_in[el.dst] == 1, 0xFFFFFFFF, (1 << 32) // np.maximum(d_in[el.dst], 1)).astype(np.uint32)
    g_gap = orc.Graph.from_edges(el, orc.W_WC)
    g_coin = orc.Graph(el.n, el.src, el.dst, orc.W_EXPLICIT, thr=thr)
    assert np.array_equal(g_gap.csr()[2], g_coin.csr()[2])  # the same thresholds, edge by edge
    N = 200_000
    res = []
    for g in (g_gap, g_coin):
        off, nodes = orc.Pool(g, orc.IC, seed=7).grow(N).arrays()
        res.append((np.diff(off), np.bincount(nodes, minlength=el.n)))
    (s_gap, c_gap), (s_coin, c_coin) = res
    assert ks_2samp(s_gap, s_coin).pvalue > 1e-3
    se = math.sqrt((s_gap.var() + s_coin.var()) / N)
    assert abs(s_gap.mean() - s_coin.mean()) < 5 * se
    top = np.argsort(-c_coin)[:50]
    z = (c_gap[top] - c_coin[top]) / np.sqrt(c_gap[top] + c_coin[top])
    assert np.abs(z).max() < 5
