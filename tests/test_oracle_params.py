"""Oracle pins for the parameter formulas (Table 1, Algorithms 1 and 4, Eqs.
"epsilon" and "set_ep", Corollary 1, the T_max expression of Sec. 5)."""
import math
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("eps,delta", [(0.1, 1e-3), (0.05, 1 / 2**20), (0.3, 0.1)])
def test_upsilon_matches_chernoff_tail(orc, eps, delta):
    # Corollary 1: T = Upsilon/mu samples make the upper-tail bound of Lemma 2 equal delta
    mu = 0.37
    T = orc.upsilon(eps, math.log(1 / delta)) / mu
    bound = math.exp(-T * mu * eps * eps / (2 + 2 * eps / 3))
    assert bound == pytest.approx(delta, rel=1e-9)


@pytest.mark.parametrize("eps", [0.02, 0.05, 0.1, 0.2, 0.3])
def test_default_eps_meets_constraint_with_equality(orc, eps):
    P = orc.params(1000, 10, eps, 1e-3, orc.SSA)
    e1, e2, e3 = P["eps1"], P["eps2"], P["eps3"]
    lhs = (1 - 1 / math.e) * (e1 + e2 + e1 * e2 + e3) / ((1 + e1) * (1 + e2))
    assert lhs == pytest.approx(eps, rel=1e-12)  # Eq. "epsilon", tight at the default
    assert e2 == e3


def test_default_eps_near_paper_example(orc):
    vals = {}
    with open(os.path.join(GOLDEN, "ssa_example_eps.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    P = orc.params(1000, 10, vals["eps"], 1e-3, orc.SSA)
    assert P["eps2"] == pytest.approx(vals["eps2"], rel=0.02)   # 0.0791 vs 2/25
    assert P["eps3"] == pytest.approx(vals["eps3"], rel=0.02)
    assert P["eps1"] == pytest.approx(vals["eps1"], rel=0.10)   # 0.0138 vs 1/78


@pytest.mark.parametrize("n,k,eps", [(2**14, 50, 0.1), (2**20, 100, 0.1), (2**23, 500, 0.05), (50, 3, 0.2)])
def test_n_max_uses_exact_binomial(orc, n, k, eps):
    # N_max (Algorithm 1 line 2) through lgamma equals the same bound with ln C(n,k)
    # from the exact integer binomial
    delta = 1.0 / n
    P = orc.params(n, k, eps, delta, orc.DSSA)
    lnC = math.log(math.comb(n, k)) if n < 10**5 else math.lgamma(n + 1) - math.lgamma(k + 1) - math.lgamma(n - k + 1)
    if n < 10**5:
        ups = orc.upsilon(eps, math.log(6 / delta) + lnC)
        ref = 8 * (1 - 1 / math.e) / (2 + 2 * eps / 3) * ups * n / k
        assert P["n_max"] == pytest.approx(ref, rel=1e-10)
    # i_max is the first power of two reaching 2 N_max / Upsilon(eps, delta/3) ...
    u3 = orc.upsilon(eps, math.log(3 / delta))
    assert 2 ** P["i_max"] >= 2 * P["n_max"] / u3 > 2 ** (P["i_max"] - 1)
    # ... so Lambda 2^(i_max-1) reaches N_max: the doubling loop ends by round i_max
    assert P["lambda"] * 2 ** (P["i_max"] - 1) >= P["n_max"]
    # D-SSA: Lambda1 = 1 + (1+eps) Lambda (Algorithm 4 line 3)
    assert P["lambda1"] == pytest.approx(1 + (1 + eps) * P["lambda"], rel=1e-15)


def test_values_of_the_four_configurations(orc):
    # Lambda, N_max, i_max, Lambda1 of the four measured workloads, computed from
    # the formulas by an independent calculation (rounded)
    table = [
        # n, k, eps, Lambda, N_max, i_max, L1_ssa, L1_dssa
        (2**14, 50, 0.1, 2806, 5.8e7, 16, 4872, 3087),
        (2**20, 100, 0.1, 3731, 5.5e9, 22, 6479, 4105),
        (2**23, 500, 0.05, 16478, 1.8e11, 25, 27374, 17303),
        (2**25, 100, 0.1, 4489, 2.4e11, 27, 7797, 4939),
    ]
    for n, k, eps, lam, nmax, imax, l1s, l1d in table:
        Ps = orc.params(n, k, eps, 1.0 / n, orc.SSA)
        Pd = orc.params(n, k, eps, 1.0 / n, orc.DSSA)
        assert round(Ps["lambda"]) == lam and Ps["i_max"] == imax
        assert Ps["n_max"] == pytest.approx(nmax, rel=0.05)
        assert round(Ps["lambda1"]) == l1s and round(Pd["lambda1"]) == l1d


def test_t_max_ratio(orc):
    # Sec. 5: T_max = 2 |R| (1+eps2)/(1-eps2) eps3^2/eps2^2; with eps2 = eps3 the ratio is 2(1+e2)/(1-e2)
    for eps in (0.1, 0.05):
        P = orc.params(1000, 10, eps, 1e-3, orc.SSA)
        e2 = P["eps2"]
        assert 2 * (1 + e2) / (1 - e2) == pytest.approx({0.1: 2.34, 0.05: 2.17}[eps], abs=0.01)
