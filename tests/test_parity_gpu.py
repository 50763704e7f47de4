"""GPU parity: the CUDA path (through the C ABI) against the oracle on the
same seeded inputs, bit-exact for every integer result (CSR, thresholds, RR
sets, counts, seed sets, coverage, Estimate-Inf T, round traces) and exactly
equal FP64 influence (the 1e-12 relative bound is the stated tolerance)."""
import itertools

import numpy as np
import pytest

import inputs
import oracle
from gpu_common import c1_edges, sorted_sets

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_1605_07990_gb300")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1605_07990_gb300 import build
    build.build()
    oracle.build()


def _pair(el, weighting=oracle.W_WC, thr=None, weight_seed=1):
    og = oracle.Graph(el.n, el.src, el.dst, weighting, thr, weight_seed)
    gg = P.ssa_load_graph(el.n, el.src, el.dst, thr, weighting, weight_seed)
    return og, gg


def _shuffled(el, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.permutation(el.m)
    return inputs.EdgeList(el.n, el.src[p].copy(), el.dst[p].copy())


@pytest.mark.parametrize("weighting", [oracle.W_WC, oracle.W_TRIVALENCY, oracle.W_EXPLICIT])
def test_graph_store(weighting):
    el = _shuffled(inputs.rmat(12, 1 << 15, seed=2))
    # duplicates and a self-loop kept as parallel edges
    el = inputs.EdgeList(el.n, np.concatenate([el.src, el.src[:50], [7]]).astype(np.int32),
                         np.concatenate([el.dst, el.dst[:50], [7]]).astype(np.int32))
    thr = None
    if weighting == oracle.W_EXPLICIT:
        thr = np.random.default_rng(3).integers(0, 2**32, el.m, dtype=np.uint64).astype(np.uint32)
    og, gg = _pair(el, weighting, thr, weight_seed=77)
    o_off, o_src, o_thr = og.csr()
    g_off, g_src, g_thr = P.ssa_graph_export(gg)
    assert np.array_equal(o_off, g_off)
    assert np.array_equal(o_src, g_src)
    assert np.array_equal(o_thr, g_thr)


def test_graph_rejects_bad_ids():
    with pytest.raises(P.SSAError):
        P.ssa_load_graph(4, np.array([0, 9], np.int32), np.array([1, 2], np.int32))


def _check_pool(og, gg, model, seed, stream, N, benefit=None):
    op = oracle.Pool(og, model, seed, stream, benefit).grow(N)
    gp = P.Pool(gg, model, seed, stream, benefit).grow(N)
    osets = op.sets()
    gsets = gp.sets()
    assert len(osets) == len(gsets) == N
    bad = [j for j in range(N) if not np.array_equal(osets[j], gsets[j])]
    assert not bad, f"{len(bad)} sets differ, first {bad[:5]}"
    return op, gp


@pytest.mark.parametrize("model", [oracle.IC, oracle.LT])
def test_rr_sets_c1(model):
    og, gg = _pair(c1_edges())
    _check_pool(og, gg, model, seed=1, stream=0, N=12_345)


def test_rr_sets_trivalency_cta_tier():
    # trivalency IC on a 2^14-node R-MAT: bimodal sizes, large sets go to the CTA tier
    el = inputs.rmat(14, 1 << 18, seed=5)
    og, gg = _pair(el, oracle.W_TRIVALENCY)
    op, gp = _check_pool(og, gg, oracle.IC, seed=9, stream=3, N=3001)
    off, _ = op.arrays()
    assert np.diff(off).max() > 512  # the CTA tier was exercised


def test_rr_sets_p1_everything_large():
    el = inputs.rmat(12, 1 << 14, seed=6)
    thr = np.full(el.m, 0xFFFFFFFF, np.uint32)
    og, gg = _pair(el, oracle.W_EXPLICIT, thr)
    _check_pool(og, gg, oracle.IC, seed=4, stream=0, N=777)


def test_rr_sets_wris():
    el = c1_edges()
    og, gg = _pair(el)
    b = inputs.zipf_benefit(el.n, 1.2, seed=3)
    for model in (oracle.IC, oracle.LT):
        _check_pool(og, gg, model, seed=5, stream=1, N=4096 + 17, benefit=b)


def test_rr_sets_empty_graph_and_isolated():
    el = inputs.edges(100, [])
    og, gg = _pair(el)
    op, gp = _check_pool(og, gg, oracle.IC, seed=1, stream=0, N=1000)
    assert all(len(s) == 1 for s in gp.sets())


def test_counts_greedy_coverage_c1(greedy_mode):
    og, gg = _pair(c1_edges())
    N = 2 * 2806
    op, gp = _check_pool(og, gg, oracle.IC, seed=1, stream=0, N=N)
    for Nsub in (2806, N, 1000):   # a batch boundary, the whole pool, and a cut inside a batch
        assert np.array_equal(op.counts(Nsub), gp.counts(Nsub).astype(np.int64))
        for k in (1, 50, 200):
            os_, og_, oc = op.max_coverage(Nsub, k)
            gs_, gg_, gc = gp.max_coverage(Nsub, k)
            assert np.array_equal(os_, gs_) and np.array_equal(og_, gg_) and oc == gc
    S = os_[:37]
    for a, b in ((0, N), (2806, N), (5, 1500)):
        assert op.coverage(a, b, S) == gp.coverage(a, b - a, S)


def test_greedy_k_equals_n(greedy_mode):
    el = inputs.rmat(6, 300, seed=1)
    og, gg = _pair(el)
    op, gp = _check_pool(og, gg, oracle.IC, seed=2, stream=0, N=500)
    os_, og_, oc = op.max_coverage(500, el.n)
    gs_, gg_, gc = gp.max_coverage(500, el.n)
    assert np.array_equal(os_, gs_) and oc == gc == 500
    assert sorted(gs_.tolist()) == list(range(el.n))


@pytest.mark.parametrize("model", [oracle.IC, oracle.LT])
def test_greedy_long_k_candidate_cache(model, greedy_mode):
    # thousands of picks on a 2^15-node graph: the greedy kernel rebuilds its
    # candidate cache many times, misses it, and falls back to full scans
    el = inputs.rmat(15, 1 << 18, seed=11)
    og, gg = _pair(el)
    N = 40_000
    op, gp = _check_pool(og, gg, model, seed=3, stream=0, N=N)
    # 20000 picks (the largest k the paper sweeps) run on past full coverage
    # into zero-gain picks, which go by smallest id
    for k in (9, 300, 3000, 20000):
        os_, og_, oc = op.max_coverage(N, k)
        gs_, gg_, gc = gp.max_coverage(N, k)
        assert np.array_equal(os_, gs_) and np.array_equal(og_, gg_) and oc == gc


def test_greedy_long_sets_queue_and_recount(greedy_mode):
    # every edge live on a 2^13-node R-MAT: sets are whole reverse-reachable
    # sets, thousands of nodes sharing one core, so covering them goes through
    # the queued-chunk path: the first pick recounts the gains, later ones drain
    el = inputs.rmat(13, 1 << 16, seed=12)
    thr = np.full(el.m, 0xFFFFFFFF, np.uint32)
    og, gg = _pair(el, oracle.W_EXPLICIT, thr)
    N = 3000
    op, gp = _check_pool(og, gg, oracle.IC, seed=6, stream=0, N=N)
    off, _ = op.arrays()
    assert (np.diff(off) > 2 * 2048).sum() > 100
    for k in (1, 5, 60):
        os_, og_, oc = op.max_coverage(N, k)
        gs_, gg_, gc = gp.max_coverage(N, k)
        assert np.array_equal(os_, gs_) and np.array_equal(og_, gg_) and oc == gc


def test_greedy_flat_gains_ties(greedy_mode):
    # an edgeless graph: every RR set is its root alone, gains are small and
    # heavily tied, so the smallest-id tie rule decides most picks
    el = inputs.edges(20_000, [])
    og, gg = _pair(el)
    N = 30_000
    op, gp = _check_pool(og, gg, oracle.IC, seed=8, stream=0, N=N)
    for k in (100, 6000):
        os_, og_, oc = op.max_coverage(N, k)
        gs_, gg_, gc = gp.max_coverage(N, k)
        assert np.array_equal(os_, gs_) and np.array_equal(og_, gg_) and oc == gc


@pytest.mark.parametrize("model", [oracle.IC, oracle.LT])
def test_estimate_inf(model):
    og, gg = _pair(c1_edges())
    op = oracle.Pool(og, model, 1, 0).grow(3000)
    S, _, _ = op.max_coverage(3000, 20)
    for lam2, t_max in ((1500.7, 10**6), (800.0, 2000), (50.2, 10**5)):
        oT, oh, _ = oracle.estimate_inf(og, model, 1, 5, S, lam2, t_max)
        gT, gh = P.ssa_estimate_inf(gg, model, 1, 5, S, lam2, t_max)
        assert (oT, oh) == (gT, gh)


@pytest.fixture(params=[1, 2], ids=["grid", "cluster"])
def greedy_mode(request):
    # the greedy kernel's two launch shapes: a cooperative grid and one thread-block cluster
    P.ssa_set_greedy_mode(request.param)
    yield request.param
    P.ssa_set_greedy_mode(0)


def _same_solution(o, g):
    assert np.array_equal(o.seeds, g.seeds)
    assert o.rounds == g.rounds
    assert o.trace == g.trace
    assert g.influence == pytest.approx(o.influence, rel=1e-12, abs=0)
    assert o.n_rr == g.n_rr


@pytest.mark.parametrize("algo,model", [(0, 0), (1, 0), (1, 1), (0, 1)])
def test_solve_c1(algo, model):
    # configuration 1 (SSA, WC-IC, k=50, eps=0.1, delta=1/n, Philox seed 1) plus the other three
    # algorithm/model pairs on the same graph
    el = c1_edges()
    og, gg = _pair(el)
    o = oracle.solve(og, algo, model, 50, 0.1, 1.0 / el.n, 1)
    g = P.ssa_solve(gg, algo, model, 50, 0.1, 1.0 / el.n, 1)
    _same_solution(o, g)


def test_solve_wris_and_trivalency():
    el = inputs.rmat(13, 1 << 16, seed=8)
    og, gg = _pair(el, oracle.W_TRIVALENCY, weight_seed=5)
    b = inputs.zipf_benefit(el.n, 1.2, seed=2)
    for algo in (0, 1):
        o = oracle.solve(og, algo, oracle.IC, 10, 0.2, 1.0 / el.n, 3, benefit=b)
        g = P.ssa_solve(gg, algo, oracle.IC, 10, 0.2, 1.0 / el.n, 3, benefit=b)
        _same_solution(o, g)


def test_solver_reuse_same_answers():
    el = c1_edges()
    gg = P.ssa_load_graph(el.n, el.src, el.dst)
    s = P.Solver(gg)
    a = s.solve(1, 0, 10, 0.1, 1.0 / el.n, 11)
    b = s.solve(1, 0, 10, 0.1, 1.0 / el.n, 11)
    c = P.ssa_solve(gg, 1, 0, 10, 0.1, 1.0 / el.n, 11)
    assert np.array_equal(a.seeds, b.seeds) and a.trace == b.trace == c.trace


def test_round_graphs_and_kept_workspaces_same_answers():
    # Each round's index, greedy and stare as one CUDA graph, patched into the
    # executable the solver keeps per round: the same seeds, traces and counts as
    # separate launches and as the oracle, over repeated solves of different
    # models, algorithms, k and WRIS on one solver (kept scratch, reused graphs)
    el = inputs.rmat(13, 1 << 16, seed=8)
    og, gg = _pair(el)
    b = inputs.zipf_benefit(el.n, 1.2, seed=2)
    plain, graphed = P.Solver(gg), P.Solver(gg).set_graphs(True)
    cases = [(1, 0, 10, 3, None), (1, 0, 10, 4, None), (1, 1, 20, 5, None), (0, 0, 10, 6, None),
             (1, 0, 50, 7, b), (0, 1, 5, 8, None), (1, 0, 10, 3, None)]
    for algo, model, k, seed, ben in cases:
        o = oracle.solve(og, algo, model, k, 0.1, 1.0 / el.n, seed, benefit=ben)
        r0 = plain.solve(algo, model, k, 0.1, 1.0 / el.n, seed, benefit=ben)
        r1 = graphed.solve(algo, model, k, 0.1, 1.0 / el.n, seed, benefit=ben)
        _same_solution(o, r0)
        _same_solution(o, r1)
        assert r0.n_rr == r1.n_rr and r0.pool_entries == r1.pool_entries
        assert r0.edge_visits == r1.edge_visits and r0.kernel_launches == r1.kernel_launches
    plain.free()
    graphed.free()


def test_bad_solve_arguments():
    el = c1_edges()
    gg = P.ssa_load_graph(el.n, el.src, el.dst, None, P.SSA_W_TRIVALENCY)
    with pytest.raises(P.SSAError):
        P.ssa_solve(gg, 1, 1, 10, 0.1, 0.01, 1)  # LT needs WC weights
    with pytest.raises(P.SSAError):
        P.ssa_solve(gg, 1, 0, 0, 0.1, 0.01, 1)
    with pytest.raises(P.SSAError):
        P.ssa_solve(gg, 1, 0, 10, 0.9, 0.01, 1)


def test_pool_cap_reports_pool_full():
    el = c1_edges()
    gg = P.ssa_load_graph(el.n, el.src, el.dst)
    with pytest.raises(P.SSAError) as e:
        P.ssa_solve(gg, 1, 0, 50, 0.1, 1.0 / el.n, 1, pool_bytes_cap=200_000)
    assert e.value.status == 3


@pytest.mark.parametrize("mid_cap,heavy", [(0, 0x7FFFFFFF), (600, 0x7FFFFFFF), (16384, 0x7FFFFFFF), (600, 8),
                                           (16384, 64)])
def test_sampler_tiers_give_identical_sets(mid_cap, heavy):
    # sets of every size class: p=1 reverse reachability on R-MAT 2^12 (up to thousands of nodes) and
    # trivalency sets (tiny or large); each hand-over size must reproduce the oracle exactly
    for el, weighting, thr in ((inputs.rmat(12, 1 << 14, seed=6), oracle.W_EXPLICIT, "p1"),
                               (inputs.rmat(14, 1 << 18, seed=5), oracle.W_TRIVALENCY, None)):
        t = np.full(el.m, 0xFFFFFFFF, np.uint32) if thr == "p1" else None
        og, gg = _pair(el, weighting, t)
        P.ssa_set_tuning(gg, mid_cap, heavy)
        op, gp = _check_pool(og, gg, oracle.IC, seed=4, stream=0, N=1500)
        seeds, _, _ = op.max_coverage(1500, 5)
        for mode_lam in (20.5, 300.0):  # hit-test mode through every tier
            assert P.ssa_estimate_inf(gg, oracle.IC, 4, 2, seeds, mode_lam, 5000) == \
                oracle.estimate_inf(og, oracle.IC, 4, 2, seeds, mode_lam, 5000)[:2]


@pytest.mark.parametrize("scale,m_draw,small_q", [(14, 1 << 18, 0), (21, 1 << 24, 0), (21, 1 << 24, 256)])
def test_wc_cta_tier_sets(scale, m_draw, small_q):
    # Weighted-cascade IC through the CTA tier's barrier-free BFS: shared-memory
    # bitmap (2^14 nodes) and global bitmap (2^21 nodes).  Handing samples over
    # at in-lists of 64 groups sends hubs through the split table; a 256-entry
    # small-CTA queue sends sets of more than 256 nodes on to the full-size CTAs.
    # Stored sets and hit-test mode both equal the oracle.
    # On the 2^21-node graph the global-bitmap warp tier (one warp per sample of
    # any size up to 2^16 nodes, visited bits in global memory) takes every
    # sample in the last two configurations.  Each configuration runs with the
    # lane tier first (sets of up to 32 nodes end there) and without it.
    el = inputs.rmat(scale, m_draw, seed=7)
    og, gg = _pair(el)
    P.ssa_set_queue_tuning(gg, small_q)
    for (mid, heavy, wg), lane in itertools.product(
            ((0, 64, 0), (0, 0x7FFFFFFF, 0), (16384, 64, 0), (0, 0x7FFFFFFF, 1), (0, 64, 1)), (0, 1)):
        P.ssa_set_tuning(gg, mid, heavy)
        P.ssa_set_warp_tier(gg, wg)
        P.ssa_set_lane_tier(gg, lane)
        op, gp = _check_pool(og, gg, oracle.IC, seed=5, stream=0, N=2000)
        seeds, _, _ = op.max_coverage(2000, 4)
        for lam in (15.5, 400.0):
            assert P.ssa_estimate_inf(gg, oracle.IC, 5, 3, seeds, lam, 3000) == \
                oracle.estimate_inf(og, oracle.IC, 5, 3, seeds, lam, 3000)[:2]
    off, _ = op.arrays()
    if small_q:
        assert np.diff(off).max() > small_q  # the full-size stage was needed
    P.ssa_set_queue_tuning(gg, 0)
    P.ssa_set_warp_tier(gg, 0)
    P.ssa_set_lane_tier(gg, 1)


def test_wc_hubs_inside_and_beyond_power_table():
    # Weighted cascade reads the gap powers of in-degrees below 2^20 from the
    # graph's table and builds those of longer in-lists itself.  Two stars feed
    # a root node: hub 1 with 2^20 - 1 in-edges (the table's last row) and hub 2
    # with 2^20 + 3 (beyond it); the root (node 0) is every set's source
    # (WRIS), and its in-list {1, 2} reaches both hubs.  Stored sets in every
    # tier (lane tier on and off) and hit-test counts equal the oracle.
    d1, d2 = (1 << 20) - 1, (1 << 20) + 3
    n = 3 + d1 + d2
    src = np.concatenate([[1, 2], np.arange(3, 3 + d1), np.arange(3 + d1, n)]).astype(np.int32)
    dst = np.concatenate([[0, 0], np.full(d1, 1), np.full(d2, 2)]).astype(np.int32)
    el = inputs.EdgeList(n, src, dst)
    og, gg = _pair(el)
    benefit = np.zeros(n, dtype=np.int64)
    benefit[0] = 1
    for lane in (1, 0):
        P.ssa_set_lane_tier(gg, lane)
        op, gp = _check_pool(og, gg, oracle.IC, seed=8, stream=0, N=3000, benefit=benefit)
    sizes = np.diff(op.arrays()[0])
    assert sizes.max() >= 3  # some sets reach a hub and take a live edge of its long in-list
    seeds = np.array([3 + d1 // 2, 3 + d1 + d2 // 2], np.int32)
    assert P.ssa_estimate_inf(gg, oracle.IC, 8, 1, seeds, 5.5, 4000, benefit=benefit) == \
        oracle.estimate_inf(og, oracle.IC, 8, 1, seeds, 5.5, 4000, benefit=benefit)[:2]
    P.ssa_set_lane_tier(gg, 1)


def test_autotune_picks_a_candidate():
    el = c1_edges()
    gg = P.ssa_load_graph(el.n, el.src, el.dst)
    cap, ms = P.ssa_autotune(gg, P.SSA_IC, 4096)
    assert cap in (0, 16384) and ms > 0
    r = P.ssa_solve(gg, 1, 0, 10, 0.1, 1.0 / el.n, 3)
    assert r.mid_cap == cap
    assert P.ssa_autotune(gg, P.SSA_LT)[0] == 0


def test_global_bitmap_ctas_and_queue_overflow():
    # n = 2^22: the CTA tier's bitmap lives in global memory (small CTAs first, full-size ones for sets
    # that outgrow the 2^20-entry small queue); with every edge live the sets are whole ancestor sets
    el = inputs.rmat(22, 1 << 25, seed=9)
    thr = np.full(el.m, 0xFFFFFFFF, np.uint32)
    og, gg = _pair(el, oracle.W_EXPLICIT, thr)
    P.ssa_set_tuning(gg, 0, 64)  # long in-lists go to the CTA tier at once
    op, gp = _check_pool(og, gg, oracle.IC, seed=2, stream=0, N=24)
    off, _ = op.arrays()
    assert np.diff(off).max() > (1 << 20)  # the full-size stage was needed
    seeds, _, _ = op.max_coverage(24, 3)
    assert P.ssa_estimate_inf(gg, oracle.IC, 2, 1, seeds, 10.5, 200) == \
        oracle.estimate_inf(og, oracle.IC, 2, 1, seeds, 10.5, 200)[:2]
    # trivalency at the same size: mostly small sets through every stage
    og2, gg2 = _pair(el, oracle.W_TRIVALENCY)
    for mid, heavy in ((0, 64), (16384, 0x7FFFFFFF)):
        P.ssa_set_tuning(gg2, mid, heavy)
        _check_pool(og2, gg2, oracle.IC, seed=3, stream=0, N=2000)


def test_lt_general_weights():
    # LT with explicit in-weights (sums <= 1, some nodes with slack): sets, greedy and full solves
    el = inputs.rmat(13, 1 << 16, seed=12)
    rng = np.random.default_rng(4)
    w = rng.uniform(0.1, 1.0, el.m)
    tot = np.zeros(el.n)
    np.add.at(tot, el.dst, w)
    frac = rng.uniform(0.6, 1.0, el.n)
    thr = np.minimum(np.floor(w * (frac / np.maximum(tot, 1e-12))[el.dst] * 2**32), 2**32 - 1).astype(np.uint32)
    og, gg = _pair(el, oracle.W_EXPLICIT, thr)
    op, gp = _check_pool(og, gg, oracle.LT, seed=6, stream=0, N=5000)
    a = op.max_coverage(5000, 30)
    b = gp.max_coverage(5000, 30)
    assert np.array_equal(a[0], b[0]) and a[2] == b[2]
    for algo in (0, 1):
        _same_solution(oracle.solve(og, algo, oracle.LT, 20, 0.1, 1.0 / el.n, 2),
                       P.ssa_solve(gg, algo, oracle.LT, 20, 0.1, 1.0 / el.n, 2))


def test_device_code_is_sm103a():
    # the runtime loaded sm_103a SASS for the library's kernels (cudaFuncGetAttributes)
    assert P.ssa_device_code_version() == (103, 103)


@pytest.mark.parametrize("scale,m_draw,weighting,seed", [(14, 1 << 17, P.SSA_W_WC, 1), (11, 1 << 15, P.SSA_W_WC, 7),
                                                         (20, 1 << 24, P.SSA_W_TRIVALENCY, 1), (3, 40, P.SSA_W_WC, 2)])
def test_gen_rmat_equals_host_generator(scale, m_draw, weighting, seed):
    # the device generator and the host input module draw the same R-MAT edges;
    # the device CSR equals the one loaded from the host edge list, bit for bit
    el = inputs.rmat(scale, m_draw, 0.57, 0.19, 0.19, seed=seed)
    gd = P.ssa_gen_rmat(scale, m_draw, 0.57, 0.19, 0.19, seed=seed, weighting=weighting, weight_seed=1)
    gh = P.ssa_load_graph(el.n, el.src, el.dst, None, weighting, 1)
    assert (gd.n, gd.m) == (el.n, el.m)
    for a, b in zip(P.ssa_graph_export(gd), P.ssa_graph_export(gh)):
        assert np.array_equal(a, b)
    if scale <= 14:
        og = oracle.Graph(el.n, el.src, el.dst, weighting, None, 1)
        off, src, thr = og.csr()
        d_off, d_src, d_thr = P.ssa_graph_export(gd)
        assert np.array_equal(off, d_off) and np.array_equal(src, d_src) and np.array_equal(thr, d_thr)
    gd.free()
    gh.free()


def test_gen_rmat_rejects_bad_arguments():
    for bad in [dict(scale=0), dict(scale=31), dict(m_draw=-1), dict(a=0.9), dict(weighting=P.SSA_W_EXPLICIT)]:
        args = dict(scale=10, m_draw=100, a=0.57, b=0.19, c=0.19, weighting=P.SSA_W_WC)
        args.update(bad)
        with pytest.raises(P.SSAError):
            P.ssa_gen_rmat(args["scale"], args["m_draw"], args["a"], args["b"], args["c"], 1, args["weighting"])
