"""Oracle pins for the stopping rules: D-SSA's eps_1, eps_2, eps_3, eps_t and
conditions D1/D2 (Algorithm 4), SSA's conditions C1/C2 (Algorithm 1) with the
Estimate-Inf result of Algorithm 3.

None of these restates the oracle's expressions.  They use:
  * a closed form: on an out-star whose every RR set holds the centre (weighted
    cascade gives each leaf one in-edge of probability 1), Cov = |R| and
    Cov_{R^c} = |R^c| at every round, so I^c = n, eps_1 = 0 and eps_2, eps_3,
    eps_t depend on eps and t only;
  * scale-free identities: with |R_t| = |R^c_t| = ceil(Lambda) 2^(t-1) and
    I^c = c n / |R^c_t|, Algorithm 4's eps_1 = Cov/c - 1,
    eps_2 = eps sqrt((1+eps) ceil(Lambda) / c) and
    eps_3 = eps sqrt((1+eps)(1-1/e-eps) ceil(Lambda) / ((1+eps/3) c)),
    whatever n or the WRIS benefit total is;
  * a second equation of the paper: with X = eps_1 + eps_2 + eps_1 eps_2,
    eps_t - eps = (1+eps_1)(1+eps_2) (LHS - eps), where LHS is the left side of
    Eq. "epsilon"; so eps_t <= eps exactly when Eq. "epsilon" holds for the
    round's three values;
  * for SSA, C2 written as a ratio of trace counts: I_hat / I_c =
    Cov T / (|R| Lambda_2), compared with 1 + eps_1, on small graphs where that
    ratio often falls between 1 + eps_1 and 1 + eps_2 (so the choice of eps in
    C2 decides the round).
Planted mistakes these catch (checked on a scratch copy of the oracle): eps_2
without its (1+eps), C2 with eps_2 in place of eps_1, eps_3 without its
(1-1/e-eps), eps_2 and eps_3 swapped in eps_t, D1 against Lambda instead of
Lambda_1."""
import math

import numpy as np
import pytest

import inputs

E1 = 1.0 - 1.0 / math.e


def star(leaves, isolated=0):
    # out-star 0 -> 1..leaves: under weighted cascade every leaf has one in-edge
    # (threshold 0xFFFFFFFF, probability 1), so every RR set rooted in the star
    # holds node 0 (IC and LT alike)
    return inputs.edges(1 + leaves + isolated, [(0, i) for i in range(1, leaves + 1)])


def eq_epsilon_lhs(e1, e2, e3):
    # Eq. "epsilon": (1-1/e) (e1 + e2 + e1 e2 + e3) / ((1+e1)(1+e2))
    return E1 * (e1 + e2 + e1 * e2 + e3) / ((1 + e1) * (1 + e2))


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("eps", [0.05, 0.1, 0.2, 0.3])
def test_dssa_all_covered_star_closed_form(orc, model, eps):
    el = star(40)
    n = el.n
    g = orc.Graph.from_edges(el, orc.W_WC)
    sol = orc.solve(g, orc.DSSA, model, 1, eps, 1.0 / n, 11)
    lam = orc.params(n, 1, eps, 1.0 / n, orc.DSSA)["lambda"]
    base = math.ceil(lam)
    assert list(sol.seeds) == [0]
    tr = sol.trace
    # round 1: c = ceil(Lambda) < 1 + (1+eps) Lambda, so D1 fails and nothing is estimated
    assert tr[0]["check_cov"] == base and tr[0]["stat"] == -1.0 and tr[0]["stop"] == 0
    assert tr[0]["eps1"] == tr[0]["eps2"] == tr[0]["eps3"] == -1.0
    # round 2: c = 2 ceil(Lambda) passes D1; with I^c = n the round's parameters are
    t = 2
    e2 = eps * math.sqrt((1 + eps) / 2 ** (t - 1))
    e3 = eps * math.sqrt((1 + eps) * (E1 - eps) / ((1 + eps / 3) * 2 ** (t - 1)))
    et = e2 * (E1 - eps) + E1 * e3
    r = tr[1]
    assert r["cov"] == r["check_cov"] == 2 * base
    assert r["eps1"] == 0.0
    assert r["eps2"] == pytest.approx(e2, rel=1e-13)
    assert r["eps3"] == pytest.approx(e3, rel=1e-13)
    assert r["stat"] == pytest.approx(et, rel=1e-13)
    # eps_t <= eps here for every eps in (0, 1-1/e): the loop stops in round 2
    assert et <= eps and r["stop"] == 1 and sol.rounds == 2
    assert sol.influence == n


def _dssa_runs(orc):
    # (graph, weighting, model, k, eps, seeds, benefit): rounds that fail D1,
    # pass D1 but fail D2, and stop, over IC and LT, uniform roots and WRIS
    cases = []
    el = inputs.rmat(11, 1 << 14, seed=5)
    cases.append((el, orc.W_WC, orc.IC, 5, 0.1, range(4), None))
    cases.append((el, orc.W_WC, orc.LT, 3, 0.2, range(4), None))
    el2 = inputs.rmat(10, 1 << 12, seed=6)
    cases.append((el2, orc.W_WC, orc.IC, 2, 0.3, range(3), inputs.zipf_benefit(el2.n, 1.2, seed=3)))
    cases.append((star(30, 30), orc.W_WC, orc.IC, 1, 0.1, range(6), None))
    for el, w, model, k, eps, seeds, benefit in cases:
        g = orc.Graph.from_edges(el, w)
        P = orc.params(el.n, k, eps, 1.0 / el.n, orc.DSSA)
        for s in seeds:
            yield el, k, eps, P, orc.solve(g, orc.DSSA, model, k, eps, 1.0 / el.n, s, benefit=benefit)


def test_dssa_round_parameters_scale_free(orc):
    seen = {"d1_fail": 0, "d2_fail": 0, "stop": 0}
    for el, k, eps, P, sol in _dssa_runs(orc):
        base = math.ceil(P["lambda"])
        for r in sol.trace:
            t, c, cov = r["t"], r["check_cov"], r["cov"]
            assert r["n_sets"] == base << (t - 1)
            capped = r["n_sets"] >= P["n_max"] or t >= P["i_max"]
            # D1: Cov_{R^c_t} >= Lambda_1 = 1 + (1+eps) Lambda (Algorithm 4, lines 3 and 9)
            d1 = c >= 1 + (1 + eps) * P["lambda"]
            if not d1:
                seen["d1_fail"] += 1
                assert r["stat"] == -1.0 and r["eps1"] == -1.0
                assert r["stop"] == int(capped)
                continue
            assert r["eps1"] == pytest.approx(cov / c - 1, rel=1e-12, abs=1e-15)
            assert r["eps2"] == pytest.approx(eps * math.sqrt((1 + eps) * base / c), rel=1e-12)
            assert r["eps3"] == pytest.approx(
                eps * math.sqrt((1 + eps) * (E1 - eps) * base / ((1 + eps / 3) * c)), rel=1e-12)
            e1, e2, e3 = r["eps1"], r["eps2"], r["eps3"]
            # eps_t ties to Eq. "epsilon" on the same three values
            assert r["stat"] - eps == pytest.approx((1 + e1) * (1 + e2) * (eq_epsilon_lhs(e1, e2, e3) - eps),
                                                    abs=1e-12)
            d2 = eq_epsilon_lhs(e1, e2, e3) <= eps
            assert (r["stat"] <= eps) == d2 or abs(r["stat"] - eps) < 1e-12
            assert r["stop"] == int(d2 or capped)
            seen["stop" if d2 else "d2_fail"] += 1
        assert sol.trace[-1]["stop"] == 1 and all(r["stop"] == 0 for r in sol.trace[:-1])
    assert min(seen.values()) >= 2, seen


@pytest.mark.parametrize("model", [0, 1])
def test_ssa_all_covered_star_closed_form(orc, model):
    # every set holds node 0: Cov = |R|, and Estimate-Inf meets node 0 in every
    # fresh set, so it stops at T = ceil(Lambda_2) and returns I_c = n Lambda_2 / T
    el = star(40)
    n, eps = el.n, 0.1
    g = orc.Graph.from_edges(el, orc.W_WC)
    P = orc.params(n, 1, eps, 1.0 / n, orc.SSA)
    sol = orc.solve(g, orc.SSA, model, 1, eps, 1.0 / n, 4)
    base = math.ceil(P["lambda"])
    first = next(t for t in range(1, 40) if (base << (t - 1)) >= P["lambda1"])  # C1 first holds
    assert sol.rounds == first
    for r in sol.trace[:-1]:
        assert r["check_cov"] == -1 and r["check_T"] == 0 and r["stop"] == 0
    r = sol.trace[-1]
    T = math.ceil(P["lambda2"])
    assert r["cov"] == r["n_sets"] and r["check_T"] == T and r["check_cov"] == T
    assert r["stat"] == pytest.approx(n * P["lambda2"] / T, rel=1e-13)
    # C2: n <= (1+eps_1) n Lambda_2 / ceil(Lambda_2) holds since ceil(Lambda_2)/Lambda_2 - 1 < 1e-3
    assert r["stop"] == 1
    assert (r["eps1"], r["eps2"], r["eps3"]) == (P["eps1"], P["eps2"], P["eps3"])


def test_ssa_condition_c2_between_eps1_and_eps2(orc):
    seen = {"window": 0, "stop": 0, "c1_fail": 0}
    for leaves, isolated, eps, seeds in [(10, 30, 0.1, range(16)), (20, 20, 0.05, range(8))]:
        el = star(leaves, isolated)
        n = el.n
        g = orc.Graph.from_edges(el, orc.W_WC)
        P = orc.params(n, 1, eps, 1.0 / n, orc.SSA)
        assert P["eps1"] < P["eps2"]
        for s in seeds:
            sol = orc.solve(g, orc.SSA, orc.IC, 1, eps, 1.0 / n, s)
            for r in sol.trace:
                capped = r["n_sets"] >= P["n_max"] or r["t"] >= P["i_max"]
                if r["cov"] < P["lambda1"]:  # C1 fails: no Estimate-Inf in this round
                    seen["c1_fail"] += 1
                    assert r["check_cov"] == -1 and r["check_T"] == 0 and r["stop"] == int(capped)
                    continue
                T = r["check_T"]
                assert T > 0  # every set rooted in the star is hit: T_max is never reached here
                assert r["stat"] == pytest.approx(n * P["lambda2"] / T, rel=1e-13)
                ratio = r["cov"] * T / (r["n_sets"] * P["lambda2"])  # I_hat / I_c
                c2 = ratio <= 1 + P["eps1"]
                assert r["stop"] == int(c2 or capped), (s, r, ratio)
                if c2:
                    seen["stop"] += 1
                elif ratio <= 1 + P["eps2"]:
                    seen["window"] += 1
    assert seen["window"] >= 5 and seen["stop"] >= 5 and seen["c1_fail"] >= 5, seen
