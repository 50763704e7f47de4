"""Thin ctypes binding of libssa (include/ssa.h): the same entry-point names,
argument marshalling only.  Every compute step runs in the library's CUDA
kernels; there is no CPU fallback -- loading fails loudly when libssa.so is
missing."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssa.so")

SSA_OK = 0
SSA_IC, SSA_LT = 0, 1
SSA_ALGO_SSA, SSA_ALGO_DSSA = 0, 1
SSA_W_WC, SSA_W_TRIVALENCY, SSA_W_EXPLICIT = 0, 1, 2
KERNEL_CLASSES = ["sample_warp", "sample_cta", "index", "greedy", "stare"]

STATUS = {0: "SSA_OK", 1: "SSA_E_ARG", 2: "SSA_E_NOMEM", 3: "SSA_E_POOL_FULL", 4: "SSA_E_CUDA",
          5: "SSA_E_TIMEOUT", 6: "SSA_E_CANCELLED", 7: "SSA_E_INTERNAL", 8: "SSA_E_NOT_READY"}


class SSAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ssa_params(C.Structure):
    _fields_ = [("algo", C.c_int), ("model", C.c_int), ("k", C.c_int32), ("eps", C.c_double),
                ("delta", C.c_double), ("seed", C.c_uint64), ("benefit", C.c_void_p),
                ("pool_bytes_cap", C.c_int64)]


class ssa_round(C.Structure):
    _fields_ = [("t", C.c_int32), ("stop", C.c_int32), ("n_sets", C.c_int64), ("cov", C.c_int64),
                ("check_cov", C.c_int64), ("check_T", C.c_int64), ("stat", C.c_double),
                ("eps1", C.c_double), ("eps2", C.c_double), ("eps3", C.c_double)]


class ssa_kstat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double)]


class ssa_result(C.Structure):
    _fields_ = [("seeds", C.c_void_p), ("trace", C.c_void_p), ("trace_cap", C.c_int32),
                ("influence", C.c_double), ("rounds", C.c_int32), ("n_rr", C.c_int64),
                ("pool_entries", C.c_int64), ("edge_visits", C.c_int64), ("node_visits", C.c_int64),
                ("cta_sets", C.c_int64), ("cta_edge_visits", C.c_int64), ("cta_node_visits", C.c_int64),
                ("cta_stored_entries", C.c_int64), ("cta_stored_sets", C.c_int64), ("draws", C.c_int64), ("cta_draws", C.c_int64),
                ("mid_cap", C.c_int32), ("heavy_groups", C.c_int32),
                ("kernel_launches", C.c_int64), ("seconds", C.c_double), ("want_kstats", C.c_int32),
                ("kstats", ssa_kstat * 5)]


class ssa_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("active", C.c_int64),
                ("pending", C.c_int64), ("bytes_budget", C.c_int64), ("bytes_in_use", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double)]


EXPORTS = {
    "ssa_status_str": (C.c_char_p, [C.c_int]),
    "ssa_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "ssa_version": (C.c_char_p, []),
    "ssa_device_code_version": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ssa_load_graph": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_uint64,
                                 C.POINTER(C.c_void_p)]),
    "ssa_gen_rmat": (C.c_int, [C.c_int32, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_int,
                               C.c_uint64, C.POINTER(C.c_void_p)]),
    "ssa_free_graph": (C.c_int, [C.c_void_p]),
    "ssa_graph_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssa_graph_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssa_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "ssa_set_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "ssa_set_wait_polls": (C.c_int, [C.c_int64]),
    "ssa_set_greedy_mode": (C.c_int, [C.c_int32]),
    "ssa_set_queue_tuning": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssa_set_warp_tier": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssa_set_lane_tier": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssa_solve": (C.c_int, [C.c_void_p, C.POINTER(ssa_params), C.POINTER(ssa_result)]),
    "ssa_solver_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    "ssa_solver_solve": (C.c_int, [C.c_void_p, C.POINTER(ssa_params), C.POINTER(ssa_result)]),
    "ssa_solver_free": (C.c_int, [C.c_void_p]),
    "ssa_solver_set_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssa_solver_set_shared": (C.c_int, [C.c_void_p, C.c_int32]),
    "ssa_pool_create": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_void_p,
                                  C.POINTER(C.c_void_p)]),
    "ssa_pool_free": (C.c_int, [C.c_void_p]),
    "ssa_pool_grow": (C.c_int, [C.c_void_p, C.c_int64]),
    "ssa_pool_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssa_pool_export": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64]),
    "ssa_pool_counts": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "ssa_max_coverage": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssa_coverage": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int32, C.c_void_p]),
    "ssa_estimate_inf": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_uint32, C.c_void_p, C.c_void_p,
                                   C.c_int32, C.c_double, C.c_int64, C.c_void_p, C.c_void_p]),
    "ssa_server_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.POINTER(C.c_void_p)]),
    "ssa_server_submit": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(ssa_params), C.POINTER(C.c_uint64)]),
    "ssa_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(ssa_result),
                                  C.POINTER(C.c_double)]),
    "ssa_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.c_void_p, C.POINTER(ssa_result),
                                  C.POINTER(C.c_double)]),
    "ssa_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ssa_serve_stats)]),
    "ssa_server_destroy": (C.c_int, [C.c_void_p]),
    "ssa_coverage_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                       C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """Load libssa.so (raises OSError when the extension is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libssa.so not built at {LIB_PATH}: run paper_1605_07990_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != SSA_OK:
        buf = C.create_string_buffer(512)
        lib().ssa_last_error(buf, 512)
        raise SSAError(status, buf.value.decode(errors="replace"))


def _ptr(a):
    return None if a is None else a.ctypes.data


def _u64(x):
    return int(x) & 0xFFFFFFFFFFFFFFFF


def ssa_version() -> str:
    return lib().ssa_version().decode()


def ssa_device_code_version():
    """(binary, ptx) architecture of the loaded device code, e.g. (103, 103)."""
    b, p = C.c_int32(), C.c_int32()
    _check(lib().ssa_device_code_version(C.byref(b), C.byref(p)))
    return b.value, p.value


# ---- graph ----
class Graph:
    """Opaque device-resident graph handle (ssa_graph*)."""

    def __init__(self, handle, n, m):
        self.h, self.n, self.m = handle, n, m

    def free(self):
        if self.h:
            _check(lib().ssa_free_graph(self.h))
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ssa_load_graph(n, src, dst, thr=None, weighting=SSA_W_WC, weight_seed=1) -> Graph:
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    thr = None if thr is None else np.ascontiguousarray(thr, dtype=np.uint32)
    h = C.c_void_p()
    _check(lib().ssa_load_graph(int(n), int(src.shape[0]), _ptr(src), _ptr(dst), _ptr(thr), int(weighting),
                                _u64(weight_seed), C.byref(h)))
    return Graph(h.value, int(n), int(src.shape[0]))


def ssa_gen_rmat(scale, m_draw, a=0.57, b=0.19, c=0.19, seed=1, weighting=SSA_W_WC, weight_seed=1) -> Graph:
    """Directed R-MAT graph generated and built on the device."""
    h = C.c_void_p()
    _check(lib().ssa_gen_rmat(int(scale), int(m_draw), float(a), float(b), float(c), _u64(seed), int(weighting),
                              _u64(weight_seed), C.byref(h)))
    n, m = C.c_int64(), C.c_int64()
    _check(lib().ssa_graph_info(h.value, C.byref(n), C.byref(m), None))
    return Graph(h.value, n.value, m.value)


def ssa_free_graph(g: Graph):
    g.free()


def ssa_graph_info(g: Graph):
    n, m, b = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().ssa_graph_info(g.h, C.byref(n), C.byref(m), C.byref(b)))
    return n.value, m.value, b.value


def ssa_graph_export(g: Graph):
    off = np.zeros(g.n + 1, dtype=np.int64)
    src = np.zeros(max(g.m, 1), dtype=np.int32)
    thr = np.zeros(max(g.m, 1), dtype=np.uint32)
    _check(lib().ssa_graph_export(g.h, _ptr(off), _ptr(src), _ptr(thr)))
    return off, src[:g.m], thr[:g.m]


def ssa_autotune(g: Graph, model=SSA_IC, pilot_samples=0):
    """Pick the IC sampler hand-over size for this graph; returns (mid_cap, pilot ms)."""
    cap, ms = C.c_int32(), C.c_double()
    _check(lib().ssa_autotune(g.h, int(model), int(pilot_samples), C.byref(cap), C.byref(ms)))
    return cap.value, ms.value


def ssa_set_tuning(g: Graph, mid_cap, heavy_groups=0x7FFFFFFF):
    _check(lib().ssa_set_tuning(g.h, int(mid_cap), int(heavy_groups)))


def ssa_set_warp_tier(g: Graph, global_bitmap=0):
    _check(lib().ssa_set_warp_tier(g.h, int(global_bitmap)))


def ssa_set_lane_tier(g: Graph, on=1):
    _check(lib().ssa_set_lane_tier(g.h, int(on)))


def ssa_set_queue_tuning(g: Graph, small_queue=0):
    _check(lib().ssa_set_queue_tuning(g.h, int(small_queue)))


def ssa_set_greedy_mode(mode=0):
    """0: cluster or grid by pool size; 1: always the cooperative grid; 2: always a cluster."""
    _check(lib().ssa_set_greedy_mode(int(mode)))


def ssa_set_wait_polls(polls=0):
    """Bound the polls of every device-side wait (0 = the default, about a second)."""
    _check(lib().ssa_set_wait_polls(int(polls)))


# ---- solve ----
@dataclass
class Result:
    seeds: np.ndarray
    influence: float
    rounds: int
    n_rr: int
    pool_entries: int
    edge_visits: int
    node_visits: int
    kernel_launches: int
    seconds: float
    cta_sets: int = 0
    cta_edge_visits: int = 0
    cta_node_visits: int = 0
    cta_stored_entries: int = 0
    cta_stored_sets: int = 0
    draws: int = 0
    cta_draws: int = 0
    mid_cap: int = 0
    heavy_groups: int = 0
    trace: list = field(default_factory=list)
    kstats: dict = field(default_factory=dict)


def _params(algo, model, k, eps, delta, seed, benefit, pool_bytes_cap):
    p = ssa_params()
    p.algo, p.model, p.k, p.eps, p.delta, p.seed = int(algo), int(model), int(k), float(eps), float(delta), _u64(seed)
    p.benefit = _ptr(benefit)
    p.pool_bytes_cap = int(pool_bytes_cap)
    return p


def _result(k, trace_cap, want_kstats):
    seeds = np.zeros(k, dtype=np.int32)
    tr = (ssa_round * trace_cap)()
    r = ssa_result()
    r.seeds = seeds.ctypes.data
    r.trace = C.cast(tr, C.c_void_p)
    r.trace_cap = trace_cap
    r.want_kstats = int(bool(want_kstats))
    return r, seeds, tr


def _unpack(r, seeds, tr):
    trace = [{"t": x.t, "stop": x.stop, "n_sets": x.n_sets, "cov": x.cov, "check_cov": x.check_cov,
              "check_T": x.check_T, "stat": x.stat, "eps1": x.eps1, "eps2": x.eps2, "eps3": x.eps3}
             for x in tr[:min(r.rounds, r.trace_cap)]]
    ks = {KERNEL_CLASSES[i]: {"launches": r.kstats[i].launches, "ms": r.kstats[i].ms} for i in range(5)}
    return Result(seeds.copy(), r.influence, r.rounds, r.n_rr, r.pool_entries, r.edge_visits, r.node_visits,
                  r.kernel_launches, r.seconds, r.cta_sets, r.cta_edge_visits, r.cta_node_visits,
                  r.cta_stored_entries, r.cta_stored_sets, r.draws, r.cta_draws, r.mid_cap, r.heavy_groups,
                  trace, ks)


def ssa_solve(g: Graph, algo, model, k, eps, delta, seed, benefit=None, pool_bytes_cap=0, want_kstats=False,
              trace_cap=64) -> Result:
    b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
    p = _params(algo, model, k, eps, delta, seed, b, pool_bytes_cap)
    r, seeds, tr = _result(k, trace_cap, want_kstats)
    _check(lib().ssa_solve(g.h, C.byref(p), C.byref(r)))
    return _unpack(r, seeds, tr)


class Solver:
    """ssa_solver*: device workspaces and a stream reused across solves."""

    def __init__(self, g: Graph, stream=None, pool_bytes_cap=0):
        h = C.c_void_p()
        _check(lib().ssa_solver_create(g.h, stream, int(pool_bytes_cap), C.byref(h)))
        self.h, self.g = h.value, g

    def solve(self, algo, model, k, eps, delta, seed, benefit=None, pool_bytes_cap=0, want_kstats=False,
              trace_cap=64) -> Result:
        b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
        p = _params(algo, model, k, eps, delta, seed, b, pool_bytes_cap)
        r, seeds, tr = _result(k, trace_cap, want_kstats)
        _check(lib().ssa_solver_solve(self.h, C.byref(p), C.byref(r)))
        return _unpack(r, seeds, tr)

    def set_graphs(self, on=True):
        """Run each round's index, greedy and stare as one CUDA graph."""
        _check(lib().ssa_solver_set_graphs(self.h, int(bool(on))))
        return self

    def set_shared(self, on=True):
        """Mark the solver as sharing the GPU with concurrent solves (cluster-shaped greedy)."""
        _check(lib().ssa_solver_set_shared(self.h, int(bool(on))))
        return self

    def free(self):
        if self.h:
            _check(lib().ssa_solver_free(self.h))
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ssa_solver_create(g, stream=None, pool_bytes_cap=0) -> Solver:
    return Solver(g, stream, pool_bytes_cap)


def ssa_solver_solve(s: Solver, *a, **kw) -> Result:
    return s.solve(*a, **kw)


def ssa_solver_free(s: Solver):
    s.free()


# ---- pools ----
class Pool:
    """ssa_pool*: RR sets of samples [0, count) of one (model, seed, stream)."""

    def __init__(self, g: Graph, model=SSA_IC, seed=1, stream=0, benefit=None):
        b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
        h = C.c_void_p()
        _check(lib().ssa_pool_create(g.h, int(model), _u64(seed), int(stream), _ptr(b), C.byref(h)))
        self.h, self.g = h.value, g

    def free(self):
        if self.h:
            _check(lib().ssa_pool_free(self.h))
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def grow(self, count):
        _check(lib().ssa_pool_grow(self.h, int(count)))
        return self

    def info(self):
        c, e, ev = C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().ssa_pool_info(self.h, C.byref(c), C.byref(e), C.byref(ev)))
        return c.value, e.value, ev.value

    def export(self, first=0, count=None):
        total = self.info()[0]
        count = total - first if count is None else count
        off = np.zeros(count + 1, dtype=np.int64)
        cap = self.info()[1]
        nodes = np.zeros(max(cap, 1), dtype=np.int32)
        _check(lib().ssa_pool_export(self.h, int(first), int(count), _ptr(off), _ptr(nodes), int(cap)))
        return off, nodes[:off[-1]]

    def set_sizes(self, first=0, count=None):
        """|R_j| for j in [first, first+count) without copying the nodes."""
        total = self.info()[0]
        count = total - first if count is None else count
        off = np.zeros(count + 1, dtype=np.int64)
        st = lib().ssa_pool_export(self.h, int(first), int(count), _ptr(off), None, 0)
        if st not in (SSA_OK, 1):  # SSA_E_ARG only reports the missing nodes buffer; off is filled
            _check(st)
        return np.diff(off)

    def sets(self, first=0, count=None, sort=True):
        off, nodes = self.export(first, count)
        out = [nodes[off[i]:off[i + 1]] for i in range(len(off) - 1)]
        return [np.sort(x) for x in out] if sort else out

    def counts(self, N):
        cnt = np.zeros(self.g.n, dtype=np.int32)
        _check(lib().ssa_pool_counts(self.h, int(N), _ptr(cnt)))
        return cnt

    def max_coverage(self, N, k):
        seeds = np.zeros(k, dtype=np.int32)
        gains = np.zeros(k, dtype=np.int64)
        cov = C.c_int64()
        _check(lib().ssa_max_coverage(self.h, int(N), int(k), _ptr(seeds), _ptr(gains), C.byref(cov)))
        return seeds, gains, cov.value

    def coverage(self, first, count, S):
        S = np.ascontiguousarray(S, dtype=np.int32)
        cov = C.c_int64()
        _check(lib().ssa_coverage(self.h, int(first), int(count), _ptr(S), int(S.shape[0]), C.byref(cov)))
        return cov.value


def ssa_pool_create(g, model=SSA_IC, seed=1, stream=0, benefit=None) -> Pool:
    return Pool(g, model, seed, stream, benefit)


def ssa_pool_grow(p: Pool, count):
    return p.grow(count)


def ssa_max_coverage(p: Pool, N, k):
    return p.max_coverage(N, k)


def ssa_coverage(p: Pool, first, count, S):
    return p.coverage(first, count, S)


def ssa_estimate_inf(g: Graph, model, seed, stream, S, lambda2, t_max, benefit=None):
    b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
    S = np.ascontiguousarray(S, dtype=np.int32)
    T, hits = C.c_int64(), C.c_int64()
    _check(lib().ssa_estimate_inf(g.h, int(model), _u64(seed), int(stream), _ptr(b), _ptr(S), int(S.shape[0]),
                                  float(lambda2), int(t_max), C.byref(T), C.byref(hits)))
    return T.value, hits.value


def ssa_coverage_noalloc(n, nodes_ptr, samp_ptr, entries, first, count, seeds_ptr, k, stream=None):
    """Allocation-free Cov over a caller-held device pool.  *_ptr are device
    addresses (e.g. torch tensor .data_ptr()); stream a cudaStream_t or None."""
    cov = C.c_int64()
    _check(lib().ssa_coverage_noalloc(int(n), nodes_ptr, samp_ptr, int(entries), int(first), int(count),
                                      seeds_ptr, int(k), C.byref(cov), stream))
    return cov.value


class Server:
    """ssa_server*: continuous-admission serving loop over resident graphs."""

    def __init__(self, graphs, slots=4, pool_bytes=0):
        arr = (C.c_void_p * len(graphs))(*[g.h for g in graphs])
        h = C.c_void_p()
        _check(lib().ssa_server_create(arr, len(graphs), int(slots), int(pool_bytes), C.byref(h)))
        self.h, self.graphs = h.value, list(graphs)
        self._k = {}

    def submit(self, graph, algo, model, k, eps, delta, seed, benefit=None):
        b = None if benefit is None else np.ascontiguousarray(benefit, dtype=np.uint32)
        p = _params(algo, model, k, eps, delta, seed, b, 0)
        t = C.c_uint64()
        _check(lib().ssa_server_submit(self.h, int(graph), C.byref(p), C.byref(t)))
        self._k[t.value] = int(k)
        return t.value

    def _take(self, fn, ticket, *extra):
        k = self._k.get(ticket, 1)  # unknown tickets are reported by the library
        r, seeds, tr = _result(k, 64, False)
        lat = C.c_double()
        st = fn(self.h, C.c_uint64(ticket), *extra, seeds.ctypes.data, C.byref(r), C.byref(lat))
        if st == 8:  # SSA_E_NOT_READY
            return None
        self._k.pop(ticket, None)
        _check(st)
        out = _unpack(r, seeds, tr)
        out.latency_s = lat.value
        return out

    def poll(self, ticket):
        return self._take(lib().ssa_server_poll, ticket)

    def wait(self, ticket, timeout_s=600.0):
        return self._take(lib().ssa_server_wait, ticket, C.c_double(timeout_s))

    def stats(self):
        st = ssa_serve_stats()
        _check(lib().ssa_server_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self.h:
            _check(lib().ssa_server_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ssa_server_create(graphs, slots=4, pool_bytes=0) -> Server:
    return Server(graphs, slots, pool_bytes)


def ssa_server_submit(s: Server, graph, *a, **kw):
    return s.submit(graph, *a, **kw)


def ssa_server_poll(s: Server, ticket):
    return s.poll(ticket)


def ssa_server_wait(s: Server, ticket, timeout_s=600.0):
    return s.wait(ticket, timeout_s)


def ssa_server_stats(s: Server):
    return s.stats()


def ssa_server_destroy(s: Server):
    s.close()
