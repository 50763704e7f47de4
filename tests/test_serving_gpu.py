"""Serving loop: queries admitted while others run give exactly the answer
they give alone (keyed randomness), the memory budget is honoured, and the
server shuts down cleanly."""
import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_1605_07990_gb300")


@pytest.fixture(scope="module")
def graphs():
    import __graft_entry__
    __graft_entry__.build()
    a = inputs.rmat(14, 1 << 17, seed=1)
    b = inputs.rmat(12, 1 << 15, seed=2)
    ga = P.ssa_load_graph(a.n, a.src, a.dst, None, P.SSA_W_WC)
    gb = P.ssa_load_graph(b.n, b.src, b.dst, None, P.SSA_W_WC)
    wa = inputs.zipf_benefit(a.n, 1.2, seed=11)
    yield (a, ga, wa), (b, gb)
    ga.free()
    gb.free()


def _queries(a, b, wa):
    rng = np.random.default_rng(5)
    qs = []
    for i in range(24):
        g = int(rng.integers(0, 2))
        n = a.n if g == 0 else b.n
        qs.append(dict(graph=g, algo=int(rng.integers(0, 2)), model=int(rng.integers(0, 2)),
                       k=int(rng.choice([1, 10, 50])), eps=float(rng.choice([0.1, 0.2])), delta=1.0 / n,
                       seed=100 + i, benefit=wa if (g == 0 and i % 2 == 0) else None))
    return qs


def test_results_same_alone_and_in_the_mix(graphs):
    (a, ga, wa), (b, gb) = graphs
    qs = _queries(a, b, wa)
    alone = []
    for q in qs:
        g = ga if q["graph"] == 0 else gb
        alone.append(P.ssa_solve(g, q["algo"], q["model"], q["k"], q["eps"], q["delta"], q["seed"],
                                 benefit=q["benefit"]))
    srv = P.Server([ga, gb], slots=4)
    tickets = [srv.submit(q["graph"], q["algo"], q["model"], q["k"], q["eps"], q["delta"], q["seed"],
                          benefit=q["benefit"]) for q in qs]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    for q, x, y in zip(qs, alone, got):
        assert np.array_equal(x.seeds, y.seeds), q
        assert x.trace == y.trace and x.influence == y.influence and x.n_rr == y.n_rr
        assert y.latency_s > 0
    assert st["completed"] == len(qs) and st["failed"] == 0 and st["active"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0


def test_budget_serialises_and_poll_not_ready(graphs):
    (a, ga, wa), _ = graphs
    # a budget below one request's footprint: requests still complete, one at a time
    srv = P.Server([ga], slots=3, pool_bytes=1 << 20)
    ts = [srv.submit(0, 1, 0, 10, 0.1, 1.0 / a.n, s) for s in range(6)]
    res = [srv.wait(t) for t in ts]
    assert all(r is not None for r in res)
    ref = P.ssa_solve(ga, 1, 0, 10, 0.1, 1.0 / a.n, 3)
    assert np.array_equal(res[3].seeds, ref.seeds)
    t = srv.submit(0, 1, 0, 10, 0.1, 1.0 / a.n, 99)
    first = srv.poll(t)  # may or may not be done yet; a finished request is released once
    if first is None:
        assert srv.wait(t) is not None
    with pytest.raises(P.SSAError):
        srv.poll(t)  # ticket already released
    srv.close()


def test_shutdown_cancels_queued(graphs):
    (a, ga, wa), _ = graphs
    srv = P.Server([ga], slots=1)
    ts = [srv.submit(0, 1, 0, 50, 0.05, 1.0 / a.n, s) for s in range(30)]
    srv.close()  # finishes the running one, cancels the rest
    with pytest.raises(P.SSAError):
        P.ssa_server_submit(srv, 0, 1, 0, 10, 0.1, 0.01, 1)
