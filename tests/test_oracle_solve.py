"""Oracle pins for the SSA (Algorithm 1) and D-SSA (Algorithm 4) drivers.

The paper prints no run, so the exact round count is "parity unpinned"; what
is pinned is the approximation guarantee (Theorems on SSA / D-SSA: with
probability >= 1-delta the returned set has I(S) >= (1-1/e-eps) OPT_k) on
graphs small enough for exact influence, plus structural facts of the loops."""
import itertools
import math

import numpy as np
import pytest

import inputs
from helpers import exact_influence_ic, exact_influence_lt_wc

TINY = inputs.edges(7, [(0, 1), (1, 2), (2, 0), (3, 0), (3, 4), (4, 5), (5, 6), (6, 4), (0, 6), (2, 5),
                        (1, 4), (6, 3)])


def _exact(model, g, S):
    off, src, thr = g.csr()
    dst = np.repeat(np.arange(g.n), np.diff(off))
    if model == 0:
        return exact_influence_ic(g.n, src, dst, thr, S)
    return exact_influence_lt_wc(g.n, src, dst, S)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("algo", [0, 1])
def test_guarantee_on_tiny_graph(orc, model, algo):
    g = orc.Graph.from_edges(TINY, orc.W_WC)
    k, eps = 2, 0.2
    infl = {S: _exact(model, g, list(S)) for S in itertools.combinations(range(g.n), k)}
    opt = max(infl.values())
    for seed in range(3):
        sol = orc.solve(g, algo, model, k, eps, 1.0 / g.n, seed)
        S = tuple(sorted(int(x) for x in sol.seeds))
        assert len(set(S)) == k
        assert infl[S] >= (1 - 1 / math.e - eps) * opt


@pytest.mark.parametrize("algo", [0, 1])
def test_loop_structure(orc, algo):
    el = inputs.rmat(12, 1 << 15, seed=1)
    g = orc.Graph.from_edges(el, orc.W_WC)
    sol = orc.solve(g, algo, orc.IC, 10, 0.1, 1.0 / el.n, 3)
    P = orc.params(el.n, 10, 0.1, 1.0 / el.n, algo)
    tr = sol.trace
    assert len(tr) == sol.rounds
    assert [r["n_sets"] for r in tr] == [math.ceil(P["lambda"]) << i for i in range(sol.rounds)]
    assert [r["stop"] for r in tr] == [0] * (sol.rounds - 1) + [1]
    last = tr[-1]
    assert sol.influence == last["cov"] * el.n / last["n_sets"]
    if algo == 1:
        # D-SSA: R_{t+1} = R_t + R^c_t, and the stop round passed D1 unless capped
        assert sol.n_rr == 2 * last["n_sets"]
        if last["n_sets"] < P["n_max"]:
            assert last["check_cov"] >= P["lambda1"] and last["stat"] <= 0.1
    else:
        if last["n_sets"] < P["n_max"]:
            assert last["cov"] >= P["lambda1"] and last["check_T"] > 0
    # same inputs, same answer
    again = orc.solve(g, algo, orc.IC, 10, 0.1, 1.0 / el.n, 3)
    assert np.array_equal(again.seeds, sol.seeds) and again.trace == sol.trace


def test_dssa_reuses_check_half(orc):
    # Algorithm 4: the sets checked in round t (R^c_t) are the second half of
    # R_{t+1}: greedy of round t+1 runs on exactly R_t + R^c_t.
    el = inputs.rmat(11, 1 << 14, seed=2)
    g = orc.Graph.from_edges(el, orc.W_WC)
    sol = orc.solve(g, 1, orc.IC, 5, 0.1, 1.0 / el.n, 8)
    if sol.rounds >= 2:
        tr = sol.trace
        pool = orc.Pool(g, orc.IC, seed=8).grow(2 * tr[-1]["n_sets"])
        for r in tr:
            seeds, gains, cov = pool.max_coverage(r["n_sets"], 5)
            assert cov == r["cov"]
            assert pool.coverage(r["n_sets"], 2 * r["n_sets"], seeds) == r["check_cov"]


def test_bad_arguments(orc):
    g = orc.Graph.from_edges(TINY, orc.W_WC)
    for bad in [dict(k=0), dict(k=8), dict(eps=0.0), dict(eps=0.7), dict(delta=1.0)]:
        a = dict(k=2, eps=0.1, delta=0.1)
        a.update(bad)
        with pytest.raises(ValueError):
            orc.solve(g, 1, 0, a["k"], a["eps"], a["delta"], 1)
