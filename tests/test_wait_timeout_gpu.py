"""Bounded device waits: failure handling tested without a GPU fault.

The greedy Max-Coverage kernel (Algorithm 2, all k picks in one cooperative
launch) synchronises its blocks with grid barriers whose waits give up after a
bounded number of polls.  Here the greedy is held to that cooperative-grid
shape (small pools otherwise run in one thread-block cluster, whose hardware
barrier needs no bound) and the bound is set to one poll, so ordinary
barriers give up: every block returns, the call reports SSA_E_TIMEOUT, and the
same CUDA context then gives the oracle's answer once the default bound is
back.  Nothing waits forever and no access changes: the kernel only returns
early."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu
SSA_E_ARG, SSA_E_TIMEOUT = 1, 5


def test_greedy_barrier_wait_gives_up_and_context_survives(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_07990_gb300 as P

    el = inputs.rmat(14, 1 << 17, seed=1)
    n = el.n
    g = P.ssa_load_graph(n, el.src, el.dst, None, P.SSA_W_WC)
    pool = P.Pool(g, P.SSA_IC, seed=5).grow(20000)
    with pytest.raises(P.SSAError) as e:
        P.ssa_set_wait_polls(-1)
    assert e.value.status == SSA_E_ARG
    try:
        P.ssa_set_greedy_mode(1)
        P.ssa_set_wait_polls(1)
        for _ in range(2):
            with pytest.raises(P.SSAError) as e:
                pool.max_coverage(20000, 50)
            assert e.value.status == SSA_E_TIMEOUT
        with pytest.raises(P.SSAError) as e:
            P.ssa_solve(g, P.SSA_ALGO_DSSA, P.SSA_IC, 50, 0.1, 1.0 / n, 3)
        assert e.value.status == SSA_E_TIMEOUT
    finally:
        P.ssa_set_wait_polls(0)
        P.ssa_set_greedy_mode(0)
    # the same context, default bound: the oracle's seeds and gains
    seeds, gains, cov = pool.max_coverage(20000, 50)
    og = orc.Graph.from_edges(el, orc.W_WC)
    opool = orc.Pool(og, orc.IC, seed=5).grow(20000)
    o_seeds, o_gains, o_cov = opool.max_coverage(20000, 50)
    assert np.array_equal(seeds, o_seeds) and np.array_equal(gains, o_gains) and cov == o_cov
    r = P.ssa_solve(g, P.SSA_ALGO_DSSA, P.SSA_IC, 50, 0.1, 1.0 / n, 3)
    o = orc.solve(og, orc.DSSA, orc.IC, 50, 0.1, 1.0 / n, 3)
    assert np.array_equal(r.seeds, o.seeds) and r.trace == o.trace
    pool.free()
    g.free()
