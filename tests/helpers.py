"""Test-side brute-force references: exact influence by enumerating live-edge
worlds, brute-force coverage / greedy, and the Chernoff bounds of Lemma 2.

These are independent statements of the definitions used to pin the oracle;
they are tiny-input only."""
from __future__ import annotations

import itertools
import math

import numpy as np

U32 = 2.0 ** 32


def edge_prob(thr: int) -> float:
    """Probability encoded by a uint32 threshold (0xFFFFFFFF = always)."""
    return 1.0 if thr == 0xFFFFFFFF else thr / U32


def reach_forward(n, live_edges, S):
    """Nodes reachable from S along live (u -> v) edges."""
    adj = [[] for _ in range(n)]
    for u, v in live_edges:
        adj[u].append(v)
    seen = set(S)
    stack = list(S)
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if v not in seen:
                seen.add(v)
                stack.append(v)
    return seen


def exact_influence_ic(n, src, dst, thr, S):
    """I(S) under IC: sum over all 2^m live-edge worlds (Sec. 2.1)."""
    m = len(src)
    ps = [edge_prob(int(t)) for t in thr]
    total = 0.0
    for mask in range(1 << m):
        pr = 1.0
        live = []
        for e in range(m):
            if mask >> e & 1:
                pr *= ps[e]
                live.append((int(src[e]), int(dst[e])))
            else:
                pr *= 1.0 - ps[e]
            if pr == 0.0:
                break
        if pr == 0.0:
            continue
        total += pr * len(reach_forward(n, live, S))
    return total


def exact_influence_lt_wc(n, src, dst, S):
    """I(S) under LT with w(u,v) = 1/d_in(v): live-edge worlds where every node
    with in-edges keeps exactly one of them, uniformly (Kempe et al.)."""
    ins = [[] for _ in range(n)]
    for e in range(len(src)):
        ins[int(dst[e])].append(int(src[e]))
    choices = [lst if lst else [None] for lst in ins]
    total = 0.0
    for pick in itertools.product(*choices):
        pr = 1.0
        live = []
        for v, u in enumerate(pick):
            if u is not None:
                pr *= 1.0 / len(ins[v])
                live.append((u, v))
        total += pr * len(reach_forward(n, live, S))
    return total


def chernoff_eps(T, mu, delta):
    """Smallest eps with exp(-T mu eps^2 / (2 + 2 eps / 3)) <= delta (Lemma 2, upper tail)."""
    L = math.log(1.0 / delta)
    a = T * mu
    # a e^2 - (2L/3) e - 2L = 0
    return ((2 * L / 3) + math.sqrt((2 * L / 3) ** 2 + 8 * a * L)) / (2 * a)


def chernoff_eps_lower(T, mu, delta):
    """eps with exp(-T mu eps^2 / 2) = delta (Lemma 2, lower tail)."""
    return math.sqrt(2 * math.log(1.0 / delta) / (T * mu))


def within_chernoff(estimate_frac, mu, T, delta=1e-6):
    up = chernoff_eps(T, mu, delta)
    lo = chernoff_eps_lower(T, mu, delta)
    return (1 - lo) * mu <= estimate_frac <= (1 + up) * mu


def coverage(sets, S):
    S = set(int(x) for x in S)
    return sum(1 for r in sets if S.intersection(int(x) for x in r))


def brute_opt_coverage(n, sets, k):
    best = -1
    for comb in itertools.combinations(range(n), k):
        best = max(best, coverage(sets, comb))
    return best


def exhaustive_greedy(n, sets, k):
    """Greedy by recomputing every marginal gain from scratch; ties -> smallest id."""
    S = []
    cur = 0
    for _ in range(k):
        best_v, best_gain = None, -1
        for v in range(n):
            if v in S:
                continue
            gain = coverage(sets, S + [v]) - cur
            if gain > best_gain:
                best_v, best_gain = v, gain
        S.append(best_v)
        cur += best_gain
    return S, cur


def ancestors(n, src, dst, root):
    """{root} plus every node with a directed path to root."""
    radj = [[] for _ in range(n)]
    for u, v in zip(src, dst):
        radj[int(v)].append(int(u))
    seen = {int(root)}
    stack = [int(root)]
    while stack:
        v = stack.pop()
        for u in radj[v]:
            if u not in seen:
                seen.add(u)
                stack.append(u)
    return seen


def exact_influence_lt_general(n, src, dst, thr, S):
    """I(S) under LT with general in-weights w_e = thr_e / 2^32 (sum <= 1 per node):
    every node keeps in-edge e with probability w_e, or none with the rest."""
    ins = [[] for _ in range(n)]
    for e in range(len(src)):
        ins[int(dst[e])].append((int(src[e]), int(thr[e]) / U32))
    choices = [lst + [(None, 1.0 - sum(w for _, w in lst))] for lst in ins]
    total = 0.0
    for pick in itertools.product(*choices):
        pr = 1.0
        live = []
        for v, (u, w) in enumerate(pick):
            pr *= w
            if u is not None:
                live.append((u, v))
        if pr > 0.0:
            total += pr * len(reach_forward(n, live, S))
    return total
