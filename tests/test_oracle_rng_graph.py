"""Oracle pins: Philox4x32-10 against its published known answers, and the
in-edge CSR / threshold encoding against brute force and the model's rules."""
import os

import numpy as np
import pytest

import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(orc, ctr, key, out):
    assert list(orc.philox4x32_10(ctr, key)) == out


def test_philox_words_uniform(orc):
    # 4 x 4096 words: each of the 16 high nibbles ~ 1/16 (loose chi-square bound)
    words = np.concatenate([orc.philox4x32_10([i, 0, 7, 3 << 28], [1, 0]) for i in range(4096)])
    hist = np.bincount(words >> 28, minlength=16)
    exp = words.size / 16
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 60  # 15 dof; p ~ 1e-7


def _brute_csr(n, src, dst):
    """In-lists ordered by (src, input position), built by plain sorting."""
    order = sorted(range(len(src)), key=lambda i: (dst[i], src[i], i))
    off = np.zeros(n + 1, dtype=np.int64)
    for i in order:
        off[dst[i] + 1] += 1
    return np.cumsum(off), [src[i] for i in order], order


def test_csr_order_and_offsets(orc):
    rng = np.random.default_rng(5)
    n, m = 37, 400
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)  # duplicates and self-loops kept
    thr = rng.integers(0, 2**32, m, dtype=np.uint64).astype(np.uint32)
    g = orc.Graph(n, src, dst, orc.W_EXPLICIT, thr)
    off, gsrc, gthr = g.csr()
    boff, bsrc, order = _brute_csr(n, list(src), list(dst))
    assert np.array_equal(off, boff)
    assert list(gsrc) == bsrc
    assert list(gthr) == [int(thr[i]) for i in order]


def test_wc_thresholds(orc):
    el = inputs.rmat(10, 1 << 13, seed=3)
    g = orc.Graph.from_edges(el, orc.W_WC)
    off, src, thr = g.csr()
    d = np.diff(off)
    for v in np.nonzero(d)[0]:
        t = thr[off[v]:off[v + 1]].astype(np.uint64)
        if d[v] == 1:
            assert t[0] == 0xFFFFFFFF  # w = 1: always live
        else:
            # w(u,v) = 1/d_in(v): t = floor(2^32 / d)
            assert np.all(t * d[v] <= 2**32) and np.all((t + 1) * d[v] > 2**32)
            # LT feasibility (Sec. 2.1): sum of in-weights <= 1
            assert t.sum() <= 2**32


def test_trivalency_thresholds(orc):
    el = inputs.rmat(12, 1 << 15, seed=4)
    g = orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=9)
    _, _, thr = g.csr()
    table = {429496729: 0.1, 42949672: 0.01, 4294967: 0.001}
    for t, p in table.items():
        assert abs(t / 2**32 - p) < 2**-32 * 2
    vals, counts = np.unique(thr, return_counts=True)
    assert set(int(v) for v in vals) == set(table)
    frac = counts / counts.sum()
    assert np.all(np.abs(frac - 1 / 3) < 0.03)
    # a different weight seed gives a different assignment
    g2 = orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=10)
    assert not np.array_equal(thr, g2.csr()[2])


def test_bad_graph_rejected(orc):
    with pytest.raises(ValueError):
        orc.Graph(4, np.array([0, 5], np.int32), np.array([1, 2], np.int32))
