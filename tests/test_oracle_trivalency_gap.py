"""Pins of the oracle's trivalency gap form (IC, Sec. 2.1; trivalency weights
w in {0.1, 0.01, 0.001}).

Each in-edge draws its class from the keyed WEIGHT draw of its rank in the
(dst, src, input position) order.  The CSR then groups every in-list by class
(0.1, 0.01, 0.001), keeping (src, position) order inside a class, and the IC
sampler walks each class's run of equal-probability edges by geometric gaps.
These tests hold that to the mathematics and to an independent restatement:

* the CSR order and thresholds against a numpy rebuild from the keying rule;
* the gap function against exact powers of q = 1 - t/2^32 for the three
  thresholds (mpmath at 200 bits);
* a star whose centre is every set's source: the live in-edges of each class
  follow Binomial(n_class, t/2^32) and every edge of a class is equally likely;
* whole RR sets on an R-MAT graph against the per-edge-coin path (explicit
  thresholds) fed the same thresholds.
"""
import math

import numpy as np
import pytest

import inputs

mpmath = pytest.importorskip("mpmath")
THR = (429496729, 42949672, 4294967)  # floor(2^32 p), p = 0.1, 0.01, 0.001


def _classes(orc, m, weight_seed):
    # the WEIGHT draw of rank e: counter (lo32(e), hi32(e), 0, 5 << 28), key = the weight seed
    key = (weight_seed & 0xFFFFFFFF, weight_seed >> 32)
    out = np.empty(m, np.int64)
    for e in range(m):
        r = orc.philox4x32_10((e & 0xFFFFFFFF, e >> 32, 0, 5 << 28), key)
        out[e] = (int(r[0]) * 3) >> 32
    return out


def test_csr_grouped_by_class(orc):
    el = inputs.rmat(9, 1 << 12, seed=21)
    ws = 7
    g = orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=ws)
    off, src, thr = g.csr()
    pos = np.arange(el.m)
    base = np.lexsort((pos, el.src, el.dst))  # (dst, src, position) order
    cls = _classes(orc, el.m, ws)            # class of each rank
    dst_b, src_b = el.dst[base], el.src[base]
    final = np.lexsort((np.arange(el.m), cls, dst_b))  # stable by (dst, class)
    assert np.array_equal(src, src_b[final])
    assert np.array_equal(thr, np.array(THR, np.uint32)[cls[final]])
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(el.dst, minlength=el.n))]))


@pytest.mark.parametrize("t", THR)
@pytest.mark.parametrize("length", [1, 2, 7, 100, 5000, 1 << 20])
def test_gap_run_thresholds_are_exact_powers(orc, t, length):
    mpmath.mp.prec = 200
    q = mpmath.mpf((1 << 32) - t) / mpmath.mpf(1 << 32)
    J = length.bit_length()
    gs = sorted({g for g in (1, 2, 3, length // 2, length - 1, length, (1 << J) - 1) if 1 <= g <= (1 << J) - 1})
    # truncated Q64 squarings: P_i is within 2^(i-64) of q^(2^i) (each squaring at most doubles the
    # error and adds 2^-64); here as an absolute margin of 2^(J+4) units of 2^-64, with a relative
    # 2^-50 on top
    two64 = mpmath.mpf(2) ** 64
    for g in gs:
        X = q ** g * two64
        tol = max(X * mpmath.mpf(2) ** -50, mpmath.mpf(2) ** (J + 4))
        lo = int(mpmath.floor(X - tol)) - 1
        hi = int(mpmath.ceil(X + tol)) + 1
        if lo >= 0:
            assert orc.gap_run(t, length, lo) >= g, (t, length, g)
        if hi < (1 << 64):
            assert orc.gap_run(t, length, hi) < g, (t, length, g)
    assert orc.gap_run(t, length, (1 << 64) - 1) == 0
    # U = 0 reaches every gap whose power survives the Q64 truncation: all of them (2^J - 1 >= length)
    # while q^(2^J - 1) is representable, else at least the largest g with q^g 2^64 above the margin
    # (for p = 0.1 the powers vanish past g of about 416, where q^g < 2^-64)
    g_rep = int(mpmath.floor(mpmath.log(mpmath.mpf(2) ** (J + 5 - 64)) / mpmath.log(q)))
    assert orc.gap_run(t, length, 0) >= min((1 << J) - 1, g_rep)
    if g_rep >= (1 << J) - 1:
        assert orc.gap_run(t, length, 0) == (1 << J) - 1 >= length


def test_star_classes_binomial(orc):
    from scipy.stats import binom, chi2

    d = 3000
    src = np.arange(1, d + 1, dtype=np.int32)
    el = inputs.EdgeList(d + 1, src, np.zeros(d, np.int32))
    g = orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=3)
    off, gsrc, thr = g.csr()
    cls_of_leaf = np.full(d + 1, -1)
    for c, t in enumerate(THR):
        cls_of_leaf[gsrc[thr == t]] = c
    benefit = np.zeros(el.n, dtype=np.int64)
    benefit[0] = 1
    N = 20000
    sets = orc.Pool(g, orc.IC, seed=13, benefit=benefit).grow(N).sets()
    assert all(s[0] == 0 for s in sets)
    for c, t in enumerate(THR):
        nc = int((cls_of_leaf == c).sum())
        p = t / 2.0 ** 32
        K = np.array([int((cls_of_leaf[s[1:]] == c).sum()) for s in sets])
        mean, sd = nc * p, math.sqrt(nc * p * (1 - p) / N)
        assert abs(K.mean() - mean) < 5 * sd, (c, K.mean(), mean)
        # P(K = 0) = q^n_c
        p0 = (1 - p) ** nc
        assert abs((K == 0).mean() - p0) < 5 * math.sqrt(max(p0 * (1 - p0), 1e-12) / N) + 1e-12
        if c == 0:
            # the whole law of the 0.1 class, pooled into cells of >= 20 expected sets
            pmf = binom.pmf(np.arange(nc + 1), nc, p)
            hist = np.bincount(K, minlength=nc + 1)
            exp, obs, ae, ao = [], [], 0.0, 0
            for k in range(nc + 1):
                ae += N * pmf[k]
                ao += hist[k]
                if ae >= 20 and N * pmf[k + 1:].sum() >= 20:
                    exp.append(ae); obs.append(ao); ae, ao = 0.0, 0
            exp.append(ae); obs.append(ao)
            exp, obs = np.array(exp), np.array(obs)
            assert ((obs - exp) ** 2 / exp).sum() < chi2.ppf(1 - 1e-4, len(exp) - 1)
            # every 0.1 edge equally likely
            inc = np.bincount(np.concatenate([s[1:] for s in sets]), minlength=d + 1)[cls_of_leaf == 0]
            e = N * p
            assert ((inc - e) ** 2 / e).sum() < chi2.ppf(1 - 1e-4, nc - 1)


def test_gap_form_matches_coins_on_rmat(orc):
    from scipy.stats import ks_2samp

    el = inputs.rmat(13, 1 << 17, seed=2)
    g_gap = orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=4)
    off, src, thr = g_gap.csr()
    dst = np.repeat(np.arange(el.n, dtype=np.int32), np.diff(off))
    g_coin = orc.Graph(el.n, src, dst, orc.W_EXPLICIT, thr=thr)  # the same edges and thresholds, per-edge coins
    N = 100_000
    res = []
    for g in (g_gap, g_coin):
        o, nodes = orc.Pool(g, orc.IC, seed=9).grow(N).arrays()
        res.append((np.diff(o), np.bincount(nodes, minlength=el.n)))
    (s_gap, c_gap), (s_coin, c_coin) = res
    assert ks_2samp(s_gap, s_coin).pvalue > 1e-3
    se = math.sqrt((s_gap.var() + s_coin.var()) / N)
    assert abs(s_gap.mean() - s_coin.mean()) < 5 * se
    top = np.argsort(-c_coin)[:50]
    z = (c_gap[top] - c_coin[top]) / np.sqrt(c_gap[top] + c_coin[top])
    assert np.abs(z).max() < 5
