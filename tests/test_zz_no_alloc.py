"""ssa_coverage_noalloc against ssa_coverage (collected last on purpose).

The allocation-free entry point serves callers that cannot allocate device
memory at call time; it keeps its scratch in one fixed device array that every
call shares.  Here it is called through the C ABI on a pool the test holds in
device memory (exported from a library pool and uploaded with torch), twice in
a row per case, and must give exactly the count ssa_coverage gives on the
library's own copy of the same pool (integer result: exact)."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_coverage_matches_ssa_coverage():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_07990_gb300 as P

    el = inputs.rmat(13, 1 << 16, seed=4)
    g = P.ssa_load_graph(el.n, el.src, el.dst, None, P.SSA_W_TRIVALENCY, 3)
    pool = P.Pool(g, P.SSA_IC, seed=3).grow(6000)
    off, nodes = pool.export()
    samp = np.repeat(np.arange(6000, dtype=np.int32), np.diff(off)).astype(np.int32)
    perm = np.random.default_rng(0).permutation(nodes.shape[0])  # entry order must not matter
    d_nodes = torch.from_numpy(nodes[perm].copy()).cuda()
    d_samp = torch.from_numpy(samp[perm].copy()).cuda()
    seeds, _, _ = pool.max_coverage(6000, 25)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(0, 6000, seeds), (1000, 2500, seeds[:7]), (5999, 1, seeds[:1]), (17, 0, seeds), (0, 6000, seeds[:0])]
    for first, count, S in cases:
        ref = pool.coverage(first, count, S)
        d_S = torch.from_numpy(np.ascontiguousarray(S, dtype=np.int32)).cuda()
        for _ in range(2):  # the shared scratch keeps the previous call's contents
            got = P.ssa_coverage_noalloc(el.n, d_nodes.data_ptr(), d_samp.data_ptr(), nodes.shape[0], first,
                                         count, d_S.data_ptr() if len(S) else None, len(S), stream)
            assert got == ref, (first, count, got, ref)
    with pytest.raises(P.SSAError):
        P.ssa_coverage_noalloc(1 << 30, d_nodes.data_ptr(), d_samp.data_ptr(), nodes.shape[0], 0, 1 << 30,
                               None, 0, stream)
