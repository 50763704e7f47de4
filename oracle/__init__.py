"""ORACLE -- test infrastructure only.

Python handle on the plain single-threaded C oracle in ``oracle.c`` (see its
header for the paper passages each part follows).  Only ``tests/``, the smoke
check and the benchmark's CPU-baseline leg may import this package; the CUDA
product path never does.  The oracle shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

IC, LT = 0, 1
SSA, DSSA = 0, 1
W_WC, W_TRIVALENCY, W_EXPLICIT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, no FP contraction so FP64 decisions follow the written order)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("n_max", C.c_double), ("i_max", C.c_int32), ("lam", C.c_double),
                ("lambda1", C.c_double), ("lambda2", C.c_double),
                ("eps1", C.c_double), ("eps2", C.c_double), ("eps3", C.c_double)]


class _Round(C.Structure):
    _fields_ = [("t", C.c_int32), ("stop", C.c_int32), ("n_sets", C.c_int64), ("cov", C.c_int64),
                ("check_cov", C.c_int64), ("check_T", C.c_int64), ("stat", C.c_double),
                ("eps1", C.c_double), ("eps2", C.c_double), ("eps3", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("influence", C.c_double), ("rounds", C.c_int32), ("n_rr", C.c_int64),
                ("pool_entries", C.c_int64), ("edge_visits", C.c_int64)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    vp, i64, u64, i32, u32, dbl = C.c_void_p, C.c_int64, C.c_uint64, C.c_int32, C.c_uint32, C.c_double
    sig = {
        "orc_philox4x32_10": (None, [vp, vp, vp]),
        "orc_wc_gap": (u32, [i64, u64]),
        "orc_graph_build": (vp, [i64, i64, vp, vp, C.c_int, vp, u64]),
        "orc_graph_free": (None, [vp]),
        "orc_graph_off": (vp, [vp]), "orc_graph_src": (vp, [vp]), "orc_graph_thr": (vp, [vp]),
        "orc_graph_n": (i64, [vp]), "orc_graph_m": (i64, [vp]),
        "orc_pool_new": (vp, [vp, C.c_int, u64, u32, vp]),
        "orc_pool_free": (None, [vp]),
        "orc_pool_grow": (None, [vp, i64]),
        "orc_pool_count": (i64, [vp]), "orc_pool_entries": (i64, [vp]),
        "orc_pool_off": (vp, [vp]), "orc_pool_nodes": (vp, [vp]),
        "orc_pool_edge_visits": (i64, [vp]),
        "orc_rr_set": (i64, [vp, C.c_int, u64, u32, u64, vp, vp]),
        "orc_sample_threads": (C.c_int, [vp, C.c_int, u64, u32, vp, u64, i64, C.c_int, vp, vp]),
        "orc_coverage": (i64, [vp, i64, i64, vp, C.c_int]),
        "orc_max_coverage": (i64, [vp, i64, C.c_int, vp, vp]),
        "orc_max_coverage_sets": (i64, [i64, i64, vp, vp, C.c_int, vp, vp]),
        "orc_counts": (None, [vp, i64, vp]),
        "orc_estimate_inf": (i64, [vp, C.c_int, u64, u32, vp, vp, C.c_int, dbl, i64, vp, vp]),
        "orc_upsilon": (dbl, [dbl, dbl]),
        "orc_params_compute": (None, [i64, C.c_int, dbl, dbl, C.c_int, vp]),
        "orc_solve": (i32, [vp, C.c_int, C.c_int, C.c_int, dbl, dbl, u64, vp, vp, vp, vp, i32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def wc_gap(d: int, U: int) -> int:
    """Dead-edge run before the next live one in a weighted-cascade in-list of
    d edges, for the 64-bit uniform U (the gap form of oracle.c)."""
    return int(_load().orc_wc_gap(d, U & 0xFFFFFFFFFFFFFFFF))


def _p(a):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


class Graph:
    """In-edge CSR with uint32 thresholds (Sec. 2, Sec. 6.1)."""

    def __init__(self, n, src, dst, weighting=W_WC, thr=None, weight_seed=1):
        L = _load()
        self._src = np.ascontiguousarray(src, dtype=np.int32)
        self._dst = np.ascontiguousarray(dst, dtype=np.int32)
        self._thr = None if thr is None else np.ascontiguousarray(thr, dtype=np.uint32)
        self.n, self.m = int(n), int(self._src.shape[0])
        h = L.orc_graph_build(self.n, self.m, _p(self._src), _p(self._dst), weighting, _p(self._thr),
                              weight_seed & 0xFFFFFFFFFFFFFFFF)
        if not h:
            raise ValueError("oracle: bad graph")
        self.h = h

    @classmethod
    def from_edges(cls, el, weighting=W_WC, thr=None, weight_seed=1):
        return cls(el.n, el.src, el.dst, weighting, thr, weight_seed)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_graph_free(self.h)
            self.h = None

    def csr(self):
        L = _load()
        off = np.ctypeslib.as_array(C.cast(L.orc_graph_off(self.h), C.POINTER(C.c_int64)), (self.n + 1,)).copy()
        if self.m == 0:
            return off, np.zeros(0, np.int32), np.zeros(0, np.uint32)
        src = np.ctypeslib.as_array(C.cast(L.orc_graph_src(self.h), C.POINTER(C.c_int32)), (self.m,)).copy()
        thr = np.ctypeslib.as_array(C.cast(L.orc_graph_thr(self.h), C.POINTER(C.c_uint32)), (self.m,)).copy()
        return off, src, thr


def benefit_prefix(benefit):
    if benefit is None:
        return None
    b = np.asarray(benefit, dtype=np.uint64)
    pre = np.zeros(b.shape[0] + 1, dtype=np.uint64)
    np.cumsum(b, out=pre[1:])
    return pre


class Pool:
    """RR sets of one stream in sample order (Definition 2)."""

    def __init__(self, g: Graph, model=IC, seed=1, stream=0, benefit=None):
        self.g = g
        self._pre = benefit_prefix(benefit)
        self.h = _load().orc_pool_new(g.h, model, seed & 0xFFFFFFFFFFFFFFFF, stream, _p(self._pre))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_pool_free(self.h)
            self.h = None

    def grow(self, count):
        _load().orc_pool_grow(self.h, count)
        return self

    @property
    def count(self):
        return _load().orc_pool_count(self.h)

    @property
    def edge_visits(self):
        return _load().orc_pool_edge_visits(self.h)

    def arrays(self):
        L = _load()
        cnt = self.count
        off = np.ctypeslib.as_array(C.cast(L.orc_pool_off(self.h), C.POINTER(C.c_int64)), (cnt + 1,)).copy()
        P = int(off[-1])
        nodes = (np.ctypeslib.as_array(C.cast(L.orc_pool_nodes(self.h), C.POINTER(C.c_int32)), (P,)).copy()
                 if P else np.zeros(0, np.int32))
        return off, nodes

    def sets(self):
        off, nodes = self.arrays()
        return [nodes[off[j]:off[j + 1]] for j in range(len(off) - 1)]

    def coverage(self, a, b, S):
        S = np.ascontiguousarray(S, dtype=np.int32)
        return int(_load().orc_coverage(self.h, a, b, _p(S), int(S.shape[0])))

    def max_coverage(self, N, k):
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        cov = _load().orc_max_coverage(self.h, N, k, _p(seeds), _p(gains))
        return seeds, gains, int(cov)

    def counts(self, N):
        cnt = np.zeros(self.g.n, dtype=np.int64)
        _load().orc_counts(self.h, N, _p(cnt))
        return cnt


def max_coverage_sets(n, sets, k):
    """Algorithm 2 on an explicit set system (list of node-id arrays)."""
    off = np.zeros(len(sets) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(x) for x in sets]) if sets else []
    nodes = (np.concatenate([np.asarray(x, dtype=np.int32) for x in sets]) if sets and off[-1] > 0
             else np.zeros(1, np.int32))
    seeds = np.zeros(k, dtype=np.int32)
    gains = np.zeros(k, dtype=np.int64)
    cov = _load().orc_max_coverage_sets(n, len(sets), _p(off), _p(nodes), k, _p(seeds), _p(gains))
    return seeds, gains, int(cov)


def rr_set(g: Graph, model, seed, stream, j, benefit=None) -> np.ndarray:
    pre = benefit_prefix(benefit)
    out = np.zeros(g.n, dtype=np.int32)
    sz = _load().orc_rr_set(g.h, model, seed & 0xFFFFFFFFFFFFFFFF, stream, j, _p(pre), _p(out))
    return out[:sz].copy()


def sample_threads(g: Graph, model, seed, stream, j0, count, threads, benefit=None):
    """RR sets [j0, j0+count) of a stream over `threads` host threads by sample
    range, counted not stored: (threads used, pool entries, edge visits)."""
    pre = benefit_prefix(benefit)
    ent = np.zeros(1, dtype=np.int64)
    ev = np.zeros(1, dtype=np.int64)
    used = _load().orc_sample_threads(g.h, model, seed & 0xFFFFFFFFFFFFFFFF, stream, _p(pre), int(j0), int(count),
                                      int(threads), _p(ent), _p(ev))
    if used < 0:
        raise ValueError("oracle: bad sample_threads arguments")
    return int(used), int(ent[0]), int(ev[0])


def estimate_inf(g: Graph, model, seed, stream, S, lambda2, t_max, benefit=None):
    """Algorithm 3: (T or 0, successes, edge visits)."""
    pre = benefit_prefix(benefit)
    S = np.ascontiguousarray(S, dtype=np.int32)
    hits = np.zeros(1, dtype=np.int64)
    ev = np.zeros(1, dtype=np.int64)
    T = _load().orc_estimate_inf(g.h, model, seed & 0xFFFFFFFFFFFFFFFF, stream, _p(pre), _p(S),
                                 int(S.shape[0]), float(lambda2), int(t_max), _p(hits), _p(ev))
    return int(T), int(hits[0]), int(ev[0])


def upsilon(eps, ln_inv_delta):
    return _load().orc_upsilon(eps, ln_inv_delta)


def params(n, k, eps, delta, algo):
    P = _Params()
    _load().orc_params_compute(n, k, eps, delta, int(algo == DSSA), C.byref(P))
    return {"n_max": P.n_max, "i_max": P.i_max, "lambda": P.lam, "lambda1": P.lambda1,
            "lambda2": P.lambda2, "eps1": P.eps1, "eps2": P.eps2, "eps3": P.eps3}


@dataclass
class Solution:
    seeds: np.ndarray
    influence: float
    rounds: int
    n_rr: int
    pool_entries: int
    edge_visits: int
    trace: list = field(default_factory=list)


def solve(g: Graph, algo, model, k, eps, delta, seed, benefit=None, max_rounds=64) -> Solution:
    """Algorithm 1 (SSA) or Algorithm 4 (D-SSA)."""
    L = _load()
    b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
    seeds = np.zeros(k, dtype=np.int32)
    res = _Result()
    tr = (_Round * max_rounds)()
    t = L.orc_solve(g.h, algo, model, k, eps, delta, seed & 0xFFFFFFFFFFFFFFFF, _p(b), _p(seeds),
                    C.byref(res), tr, max_rounds)
    if t < 0:
        raise ValueError("oracle: bad solve arguments")
    trace = [{"t": r.t, "stop": r.stop, "n_sets": r.n_sets, "cov": r.cov, "check_cov": r.check_cov,
              "check_T": r.check_T, "stat": r.stat, "eps1": r.eps1, "eps2": r.eps2, "eps3": r.eps3}
             for r in tr[:min(t, max_rounds)]]
    return Solution(seeds, res.influence, res.rounds, res.n_rr, res.pool_entries, res.edge_visits, trace)
