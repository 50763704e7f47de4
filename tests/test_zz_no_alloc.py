"""ssa_coverage_noalloc against ssa_coverage and the oracle's Cov (collected last
on purpose).

The allocation-free entry point serves callers that cannot allocate device
memory at call time; it keeps its scratch in one fixed device array that every
call shares.  Here it is called through the C ABI on a pool the test holds in
device memory (exported from a library pool and uploaded with torch), twice in
a row per case.  It must give exactly the count that ssa_coverage gives on the
library's own copy of the same pool, and the count the oracle gives on its own
pool of the same sets (Eq. 1; integer result: exact).  Ids outside [0, n) are
rejected by the device's own bounds checks (nothing is read out of bounds), and
the next call is exact again: the shared flag does not stick."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_coverage_matches_ssa_coverage_and_oracle(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_07990_gb300 as P

    el = inputs.rmat(13, 1 << 16, seed=4)
    g = P.ssa_load_graph(el.n, el.src, el.dst, None, P.SSA_W_TRIVALENCY, 3)
    pool = P.Pool(g, P.SSA_IC, seed=3).grow(6000)
    opool = orc.Pool(orc.Graph.from_edges(el, orc.W_TRIVALENCY, weight_seed=3), orc.IC, seed=3).grow(6000)
    off, nodes = pool.export()
    samp = np.repeat(np.arange(6000, dtype=np.int32), np.diff(off)).astype(np.int32)
    perm = np.random.default_rng(0).permutation(nodes.shape[0])  # entry order must not matter
    d_nodes = torch.from_numpy(nodes[perm].copy()).cuda()
    d_samp = torch.from_numpy(samp[perm].copy()).cuda()
    seeds, _, _ = pool.max_coverage(6000, 25)
    stream = torch.cuda.current_stream().cuda_stream

    def noalloc(first, count, S, n=el.n, d_n=d_nodes, d_s=d_samp):
        d_S = torch.from_numpy(np.ascontiguousarray(S, dtype=np.int32)).cuda()
        return P.ssa_coverage_noalloc(n, d_n.data_ptr(), d_s.data_ptr(), d_n.shape[0], first, count,
                                      d_S.data_ptr() if len(S) else None, len(S), stream)

    cases = [(0, 6000, seeds), (1000, 2500, seeds[:7]), (5999, 1, seeds[:1]), (17, 0, seeds), (0, 6000, seeds[:0])]
    for first, count, S in cases:
        ref = pool.coverage(first, count, S)
        assert ref == opool.coverage(first, first + count, S)
        for _ in range(2):  # the shared scratch keeps the previous call's contents
            got = noalloc(first, count, S)
            assert got == ref, (first, count, got, ref)
    with pytest.raises(P.SSAError):
        P.ssa_coverage_noalloc(1 << 30, d_nodes.data_ptr(), d_samp.data_ptr(), nodes.shape[0], 0, 1 << 30,
                               None, 0, stream)
    # a seed id equal to n, then a pool entry holding node n inside the counted window:
    # each call is rejected, and a valid call right after is exact
    with pytest.raises(P.SSAError):
        noalloc(0, 6000, np.array([1, el.n], dtype=np.int32))
    bad = nodes[perm].copy()
    j = int(np.flatnonzero(samp[perm] == 1500)[0])
    bad[j] = el.n
    d_bad = torch.from_numpy(bad).cuda()
    with pytest.raises(P.SSAError):
        noalloc(1000, 1000, seeds, d_n=d_bad)
    assert noalloc(0, 6000, seeds) == pool.coverage(0, 6000, seeds)
    assert noalloc(1000, 1000, seeds) == pool.coverage(1000, 1000, seeds)
