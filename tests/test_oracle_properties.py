"""Property tests of the oracle on random small inputs (hypothesis).

- IC: every RR set is the set of nodes that reach the sample's root through
  live edges (Definition 2). Here the live-edge world is rebuilt edge by edge
  from the keying rule: Philox4x32-10 with key (lo32(seed), hi32(seed)) and
  counter (lo32(x), hi32(x), lo32(j), purpose<<28 | stream<<20 | hi bits of j).
  Reachability then comes from a plain graph search, not from the oracle's BFS.
- LT: the live-edge world keeps at most one in-edge per node (Sec. 2.1). The
  kept edge is rebuilt from the same keying: weighted cascade takes edge
  floor(r * d_in / 2^32); general weights take the first edge whose running
  threshold sum passes r. The RR set is again the reverse-reachable set in
  that world.
- WRIS (Sec. 6.3.1): a root is never a zero-benefit node.
- Algorithm 2 on random set systems equals a greedy that recomputes every
  marginal gain from scratch, with the smallest id winning ties.
- Algorithm 3 stops at the first prefix of the stream whose hit count reaches
  Lambda_2.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

M32 = 0xFFFFFFFF
ALWAYS = 0xFFFFFFFF
ROOT, IC_COIN, LT_PICK = 1, 2, 3
SETTINGS = settings(max_examples=150, deadline=None, suppress_health_check=[HealthCheck.too_slow])


def keyed(orc, seed, purpose, stream, j, x):
    ctr = [x & M32, (x >> 32) & M32, j & M32, (purpose << 28) | ((stream & 0xFF) << 20) | ((j >> 32) & 0xFFFFF)]
    return [int(w) for w in orc.philox4x32_10(ctr, [seed & M32, (seed >> 32) & M32])]


def reverse_reachable(n, live_edges, root):
    """Nodes with a path to root over the given (u, v) edges."""
    preds = {v: [] for v in range(n)}
    for u, v in live_edges:
        preds[v].append(u)
    seen, stack = {root}, [root]
    while stack:
        v = stack.pop()
        for u in preds[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return sorted(seen)


@st.composite
def small_graph(draw, max_n=9, max_m=18):
    n = draw(st.integers(1, max_n))
    m = draw(st.integers(0, max_m))
    edges = [(draw(st.integers(0, n - 1)), draw(st.integers(0, n - 1))) for _ in range(m)]
    return n, edges


keys = st.tuples(st.integers(0, 2**64 - 1), st.integers(0, 255), st.integers(0, 2**44))


@SETTINGS
@given(small_graph(), st.data(), keys)
def test_ic_rr_set_is_reverse_reachable_in_keyed_world(orc, ng, data, key):
    n, edges = ng
    seed, stream, j = key
    thr_in = [data.draw(st.sampled_from([0, ALWAYS, 1 << 31]) | st.integers(0, M32)) for _ in edges]
    src = np.array([u for u, _ in edges], np.int32)
    dst = np.array([v for _, v in edges], np.int32)
    g = orc.Graph(n, src, dst, orc.W_EXPLICIT, np.array(thr_in, np.uint32))
    off, csrc, cthr = g.csr()
    live = []
    for v in range(n):
        for e in range(off[v], off[v + 1]):
            coin = keyed(orc, seed, IC_COIN, stream, j, e >> 2)[e & 3]
            if cthr[e] == ALWAYS or coin < cthr[e]:
                live.append((int(csrc[e]), v))
    root = (keyed(orc, seed, ROOT, stream, j, 0)[0] * n) >> 32
    want = reverse_reachable(n, live, root)
    assert orc.rr_set(g, orc.IC, seed, stream, j).tolist() == want


@SETTINGS
@given(small_graph(), st.data(), keys, st.booleans())
def test_lt_rr_set_is_reverse_reachable_in_keyed_world(orc, ng, data, key, general):
    n, edges = ng
    seed, stream, j = key
    src = np.array([u for u, _ in edges], np.int32)
    dst = np.array([v for _, v in edges], np.int32)
    if general:
        # per-node weights with sum <= 1: each of the d_in thresholds at most 2^32 / d_in
        d_in = np.bincount(dst, minlength=n) if len(edges) else np.zeros(n, np.int64)
        thr = np.array([data.draw(st.integers(0, (1 << 32) // int(d_in[v]))) for v in dst.tolist()], np.uint64)
        g = orc.Graph(n, src, dst, orc.W_EXPLICIT, np.minimum(thr, M32).astype(np.uint32))
    else:
        g = orc.Graph(n, src, dst, orc.W_WC)
    off, csrc, cthr = g.csr()
    kept = []
    for v in range(n):
        d = int(off[v + 1] - off[v])
        if d == 0:
            continue
        r = keyed(orc, seed, LT_PICK, stream, j, v)[0]
        if general:
            cum, pick = 0, None
            for e in range(off[v], off[v + 1]):
                cum += int(cthr[e])
                if r < cum:
                    pick = e
                    break
        else:
            pick = int(off[v]) + ((r * d) >> 32)
        if pick is not None:
            kept.append((int(csrc[pick]), v))
    root = (keyed(orc, seed, ROOT, stream, j, 0)[0] * n) >> 32
    want = reverse_reachable(n, kept, root)
    assert orc.rr_set(g, orc.LT, seed, stream, j).tolist() == want


@SETTINGS
@given(st.lists(st.integers(0, 5), min_size=1, max_size=12), st.integers(0, 2**32), st.integers(0, 255))
def test_wris_root_has_positive_benefit(orc, benefit, seed, stream):
    if sum(benefit) == 0:
        benefit[0] = 1
    n = len(benefit)
    g = orc.Graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32), orc.W_WC)
    b = np.array(benefit, np.uint32)
    for j in range(20):
        R = orc.rr_set(g, orc.IC, seed, stream, j, benefit=b)
        assert len(R) == 1 and benefit[int(R[0])] > 0


def recompute_greedy(n, sets, k):
    covered = [False] * len(sets)
    picked, gains = [], []
    for _ in range(k):
        best, best_gain = None, -1
        for v in range(n):
            if v in picked:
                continue
            gain = sum(1 for i, s in enumerate(sets) if not covered[i] and v in s)
            if gain > best_gain:
                best, best_gain = v, gain
        picked.append(best)
        gains.append(best_gain)
        for i, s in enumerate(sets):
            if best in s:
                covered[i] = True
    return picked, gains


@SETTINGS
@given(st.integers(1, 10).flatmap(lambda n: st.tuples(
    st.just(n),
    st.lists(st.sets(st.integers(0, n - 1), min_size=1, max_size=n), min_size=0, max_size=25),
    st.integers(1, n))))
def test_max_coverage_equals_recompute_greedy(orc, case):
    n, sets, k = case
    seeds, gains, cov = orc.max_coverage_sets(n, [np.array(sorted(s), np.int32) for s in sets], k)
    want_seeds, want_gains = recompute_greedy(n, [set(s) for s in sets], k)
    assert seeds.tolist() == want_seeds
    assert gains.tolist() == want_gains
    assert cov == sum(want_gains)


@st.composite
def sorted_unique_graph(draw, max_n=8):
    """Edges already in in-edge CSR order (by head, then tail), so that the
    input position of an edge is its CSR position."""
    n = draw(st.integers(2, max_n))
    pairs = draw(st.sets(st.tuples(st.integers(0, n - 1), st.integers(0, n - 1)), min_size=1, max_size=16))
    edges = sorted(pairs, key=lambda e: (e[1], e[0]))
    return n, edges


@SETTINGS
@given(sorted_unique_graph(), st.data(), keys)
def test_ic_coin_equal_to_threshold_is_dead(orc, ng, data, key):
    # thresholds set to the edge's own coin (dead: live needs coin < thr) or
    # one above it (live), so the strict inequality decides every edge
    n, edges = ng
    seed, stream, j = key
    src = np.array([u for u, _ in edges], np.int32)
    dst = np.array([v for _, v in edges], np.int32)
    coins = [keyed(orc, seed, IC_COIN, stream, j, e >> 2)[e & 3] for e in range(len(edges))]
    up = [data.draw(st.booleans()) and c < ALWAYS - 1 for c in coins]
    thr = np.array([c + 1 if u else min(c, ALWAYS - 1) for c, u in zip(coins, up)], np.uint32)
    g = orc.Graph(n, src, dst, orc.W_EXPLICIT, thr)
    off, csrc, cthr = g.csr()
    assert csrc.tolist() == src.tolist() and cthr.tolist() == thr.tolist()
    live = [(int(src[e]), int(dst[e])) for e in range(len(edges)) if coins[e] < int(thr[e])]
    root = (keyed(orc, seed, ROOT, stream, j, 0)[0] * n) >> 32
    assert orc.rr_set(g, orc.IC, seed, stream, j).tolist() == reverse_reachable(n, live, root)


@SETTINGS
@given(st.integers(2, 6), st.data(), keys)
def test_lt_running_sum_equal_to_draw_passes_on(orc, d, data, key):
    # a star of d in-edges into node 0 (tails 1..d); the running threshold sum
    # reaches the draw exactly after edge i, so the pick is edge i + 1 (none
    # after the last edge)
    seed, stream, j = key
    n = d + 1
    src = np.arange(1, n, dtype=np.int32)
    dst = np.zeros(d, np.int32)
    r = keyed(orc, seed, LT_PICK, stream, j, 0)[0]
    i = data.draw(st.integers(0, d - 1))
    head = [data.draw(st.integers(0, r // (2 * d))) for _ in range(i)]
    t = head + [r - sum(head)] + [data.draw(st.integers(1, 1000)) for _ in range(d - 1 - i)]
    assert sum(t) <= 1 << 32
    g = orc.Graph(n, src, dst, orc.W_EXPLICIT, np.array(t, np.uint32))
    tail = i + 2 if i + 1 < d else None  # edge i + 1 has tail i + 2
    root = (keyed(orc, seed, ROOT, stream, j, 0)[0] * n) >> 32
    want = [root] if root != 0 or tail is None else [0, tail]
    assert orc.rr_set(g, orc.LT, seed, stream, j).tolist() == want


@SETTINGS
@given(small_graph(max_n=7, max_m=12), st.data(), keys, st.sampled_from([0, 1]))
def test_estimate_inf_is_first_prefix_reaching_lambda2(orc, ng, data, key, model):
    # Algorithm 3: T is the first prefix of the sample stream whose hit count
    # reaches Lambda_2 (0 when T_max sets do not), computed here from the RR
    # sets one by one
    n, edges = ng
    seed, stream, _ = key
    src = np.array([u for u, _ in edges], np.int32)
    dst = np.array([v for _, v in edges], np.int32)
    g = orc.Graph(n, src, dst, orc.W_WC)
    S = sorted(data.draw(st.sets(st.integers(0, n - 1), min_size=1, max_size=n)))
    lam2 = data.draw(st.floats(0.5, 12.0))
    t_max = data.draw(st.integers(1, 40))
    T, hits, _ = orc.estimate_inf(g, model, seed, stream, np.array(S, np.int32), lam2, t_max)
    cov, want_T = 0, 0
    for j in range(t_max):
        cov += bool(set(orc.rr_set(g, model, seed, stream, j).tolist()) & set(S))
        if cov >= lam2:
            want_T = j + 1
            break
    assert (T, hits) == (want_T, cov)
