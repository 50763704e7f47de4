"""Benchmark: RR sets/s of whole SSA / D-SSA solves on a resident synthetic R-MAT graph.

One step = one complete solve on the GPU: RR sampling of every doubling round,
the node->set index, greedy Max-Coverage, the stare check and the host FP64
stopping rule.  Default workload (the billion-edge configuration): plain SSA
(Algorithm 1), IC with weighted-cascade weights w = 1/d_in, directed R-MAT on
2^25 nodes from 1.3e9 draws (a,b,c,d = 0.57,0.19,0.19,0.05; duplicates and
self-loops removed: 1,263,509,823 edges), k=100, eps=0.1, delta=1/n; each step
draws a fresh Philox seed.  The D-SSA trivalency workload on 2^20 nodes / 2^24
draws is measured in the same run and reported under "extra".

value = RR sets generated / device time of the timed steps (inputs resident).
e2e = the same metric through the C ABI from pinned host edge arrays: graph
upload, device CSR build, solve and seeds back, every step.
roofline = the dominant kernel class against its real bound (see roofline()).
cpu_baseline = the oracle as it stands on the host cores: the sampling phase on
one thread and over all cores (by sample range), then Max-Coverage and the
stare count over the one-thread sample.

--impl reference times the oracle on the host cores on a bounded sample of the
same workload per step.  Multi-GPU (torchrun): independent replicas, one per
rank (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (scale, m_draw, weighting, algo, model, k, eps)
    "ssa_ic_wc_rmat25_m1.3G_k100": (25, 1_300_000_000, 0, 0, 0, 100, 0.1),
    "dssa_ic_trivalency_rmat20_m16M_k100": (20, 1 << 24, 1, 1, 0, 100, 0.1),
    "ssa_ic_wc_rmat14_m128K_k50": (14, 1 << 17, 0, 0, 0, 50, 0.1),
    "dssa_lt_wc_rmat23_m128M_k500": (23, 1 << 27, 0, 1, 1, 500, 0.05),
    # a tenth of the billion-edge graph, same model and weights: small enough for ncu captures
    "ssa_ic_wc_rmat23_m128M_k100": (23, 1 << 27, 0, 0, 0, 100, 0.1),
}
DEFAULT = "ssa_ic_wc_rmat25_m1.3G_k100"
EXTRA = "dssa_ic_trivalency_rmat20_m16M_k100"
METRIC, UNIT = "RR sets/s", "RR sets/s"
WEIGHTS = ["weighted-cascade", "trivalency"]

# ALU roofline of the IC samplers with edge records (trivalency, explicit
# weights).  Each coin comes from one Philox4x32-10 draw per 4-edge group: 10
# rounds of two 32x32->64 multiplies and two three-input XORs, 40 thread
# instructions at least.  At one warp instruction per SM sub-partition per
# clock (4 per SM) the GPU issues at most
#   SMs x 4 x clock x 32 lanes / 40 draws per second.
# The weighted-cascade sampler walks in-lists by geometric gaps (one draw per
# two gaps, no per-edge coins) and is reported against HBM instead.
PHILOX_MIN_INSTR = 40

# DRAM bytes per unit of work from ncu captures of the sampler kernels
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by workload and kernel
# class, valid only for the kernel sources they were taken on (hash of
# csrc/sample.cu, csrc/device.cuh, csrc/kernels.h); any other build reports
# traffic null.
TRAFFIC = {
    # 2^23-node capture (profiles/sample_warp_wcg_wc_ic_rmat23.md): 14.14 GB of DRAM traffic over
    # 47,589,152 node visits for the lane and warp tiers of a 2M-set grow, scaled to the 2^25-node
    # workload by its node visits (the traffic is four to five random sector touches per visit)
    ("ssa_ic_wc_rmat25_m1.3G_k100", "sample_warp"): {"src": "856e006a6deed4db", "bytes_per_node_visit": 297.2},
    ("ssa_ic_wc_rmat23_m128M_k100", "sample_warp"): {"src": "856e006a6deed4db", "bytes_per_node_visit": 297.2},
}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("sample.cu", "device.cuh", "kernels.h"):
        with open(os.path.join(ROOT, "paper_1605_07990_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def replica_seed(rank: int, step: int) -> int:
    """Philox seed of a timed step: each rank is an independent replica, so
    ranks and steps never share a seed (warm-up steps use 10000 + w + 1000 rank)."""
    return 1 + step + 1000 * rank


def reduce_over_ranks(ms: float, counts, device) -> tuple:
    """Job-level timing and totals over the process group: the slowest rank's
    time and the sums of the per-rank counts (RR sets, edge visits, node visits)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(x) for x in c.tolist()]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (200 ms) run during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id, self.proc, self.lines = gpu_id, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


def make_graph_inputs(name):
    import inputs
    scale, m_draw, weighting, algo, model, k, eps = WORKLOADS[name]
    el = inputs.rmat(scale, m_draw, 0.57, 0.19, 0.19, seed=1)
    return el, weighting, algo, model, k, eps


def sampler_model(weighting, model):
    if model == 1:
        return "lt"
    return "ic_wc" if weighting == 0 else "ic_records"


def roofline(kind, dom, ks, results, sm_count, clock_mhz, name, hbm_peak, hbm_kind):
    """Roofline of the dominant kernel class (a sampler tier).

    Weighted-cascade IC (gap walk): bound "hbm".  Algorithmic bytes per unit:
    16 per visited node (two CSR offsets), 8 per live edge taken (its record;
    one per visited node but the root), 8 per stored pool entry (node,
    sample), 12 per stored set (start, length), 1 per hit-tested set.  No
    per-edge bytes: the gaps need only the in-degree.
    Edge records (trivalency, explicit): bound "alu" in Philox draws/s against
    PHILOX_MIN_INSTR, with 8 per examined in-edge in the HBM side figure."""
    if dom not in ("sample_cta", "sample_warp") or kind == "lt" or ks[dom]["ms"] <= 0:
        return None
    cta = dom == "sample_cta"
    draws = sum((r.cta_draws if cta else r.draws - r.cta_draws) for r in results)
    ev = sum((r.cta_edge_visits if cta else r.edge_visits - r.cta_edge_visits) for r in results)
    nv = sum((r.cta_node_visits if cta else r.node_visits - r.cta_node_visits) for r in results)
    sets = sum((r.cta_sets if cta else r.n_rr - r.cta_sets) for r in results)
    st_e = sum((r.cta_stored_entries if cta else r.pool_entries - r.cta_stored_entries) for r in results)
    st_s = sum((r.cta_stored_sets if cta else r.trace[-1]["n_sets"] - r.cta_stored_sets) for r in results)
    sec = ks[dom]["ms"] / 1000.0
    launches = max(1, ks[dom]["launches"])
    tr = TRAFFIC.get((name, dom))
    traffic = None
    if tr and tr["src"] == kernel_source_hash():
        traffic = tr["bytes_per_node_visit"] * nv / launches
    common = {"kernel": dom, "traffic": traffic,
              # the DRAM rate the measured traffic implies over the class's CUDA-event time
              "traffic_gbs": traffic / (ks[dom]["ms"] / launches / 1000.0) / 1e9 if traffic is not None else None,
              "avg_launch_ms": ks[dom]["ms"] / launches,
              "node_visits_per_launch": nv / launches, "node_visits_per_s": nv / sec,
              "philox_draws_per_s": draws / sec}
    if kind == "ic_wc":
        abytes = 16 * nv + 8 * max(nv - sets, 0) + 8 * st_e + 12 * st_s + max(sets - st_s, 0)
        ach = abytes / sec / 1e9
        return {**common, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": hbm_kind,
                "algorithmic_bytes_per_launch": abytes / launches,
                "implied_edge_visits_per_s": ev / sec}
    peak = sm_count * 4 * clock_mhz * 1e6 * 32 / PHILOX_MIN_INSTR
    ach = draws / sec
    abytes = 8 * ev + 16 * nv + 8 * st_e + 12 * st_s + max(sets - st_s, 0)
    return {**common, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Philox draws/s",
            "frac": ach / peak,
            "peak_source": f"derived: {sm_count} SMs x 4 issue slots x {clock_mhz:.0f} MHz x 32 lanes / "
                           f"{PHILOX_MIN_INSTR} instructions per Philox4x32-10 draw",
            "draws_per_launch": draws / launches, "edge_visits_per_launch": ev / launches,
            "hbm": {"algorithmic_bytes_per_launch": abytes / launches, "algorithmic_gbs": abytes / sec / 1e9,
                    "peak_gbs": hbm_peak, "frac": abytes / sec / 1e9 / hbm_peak, "peak_source": hbm_kind}}


def run_solves(P, solver, name, steps, warmup, seed_of, stream, torch):
    scale, m_draw, weighting, algo, model, k, eps = WORKLOADS[name]
    n = 1 << scale
    delta = 1.0 / n
    for w in range(warmup):
        solver.solve(algo, model, k, eps, delta, 10_000 + w + seed_of(0) - 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    e0.record(stream)
    for s in range(steps):
        results.append(solver.solve(algo, model, k, eps, delta, seed_of(s), want_kstats=True))
    e1.record(stream)
    torch.cuda.synchronize()
    return results, e0.elapsed_time(e1)


def summarise(P, name, results, ms, sm_count, clock_mhz):
    scale, m_draw, weighting, algo, model, k, eps = WORKLOADS[name]
    sec = ms / 1000.0
    rr = sum(r.n_rr for r in results)
    stored = sum(r.trace[-1]["n_sets"] for r in results)
    ks = {c: {"launches": sum(r.kstats[c]["launches"] for r in results),
              "ms": sum(r.kstats[c]["ms"] for r in results)} for c in P.binding.KERNEL_CLASSES}
    dom = max(ks, key=lambda c: ks[c]["ms"])
    hbm_peak, hbm_kind = peaks()
    roof = roofline(sampler_model(weighting, model), dom, ks, results, sm_count, clock_mhz, name, hbm_peak,
                    hbm_kind)
    return {
        "value": rr / sec, "ms_per_step": ms / len(results),
        "edge_visits_per_s": sum(r.edge_visits for r in results) / sec,
        "node_visits_per_s": sum(r.node_visits for r in results) / sec,
        "philox_draws_per_s": sum(r.draws for r in results) / sec,
        "rr_sets_per_solve": rr / len(results),
        # SSA's Estimate-Inf sets and D-SSA's final check half are sampled in hit-test mode
        # (each RR set stops at its first seed) and not stored; they count as drawn
        "rr_sets_stored_per_solve": stored / len(results),
        "rr_sets_hit_tested_per_solve": (rr - stored) / len(results),
        "rounds": [r.rounds for r in results], "kernel_ms": ks, "dominant": dom,
        "gpu_launches": sum(r.kernel_launches for r in results), "roofline": roof,
    }


class OracleGraph(threading.Thread):
    """The oracle's CSR of the workload, built on a host thread (the C call
    releases the GIL) while the GPU steps run."""

    def __init__(self, el, weighting):
        super().__init__(daemon=True)
        self.el, self.weighting, self.g, self.seconds, self.error = el, weighting, None, 0.0, None

    def run(self):
        try:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            self.g = oracle.Graph(self.el.n, self.el.src, self.el.dst, self.weighting, None, 1)
            self.seconds = time.perf_counter() - t0
        except Exception as e:  # reported in the bench line
            self.error = repr(e)


def cpu_baseline(og, t_graph, el, model, k, seed, budget_s):
    """The oracle as it stands on the host cores: the sampling phase of the step-0
    solve's stream on one thread for about budget_s, the same number of sets per
    thread over all cores (by sample range), then Max-Coverage (Algorithm 2) and
    the stare count (Eq. 1) over the one-thread sample."""
    import oracle
    pool = oracle.Pool(og, model, seed, 0)
    t0 = time.perf_counter()
    count, chunk = 0, 4
    while time.perf_counter() - t0 < budget_s:
        count += chunk
        pool.grow(count)
        chunk = min(chunk * 2, 64)
    t_one = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    used, _, _ = oracle.sample_threads(og, model, seed, 0, count, count * cores, cores)
    t_all = time.perf_counter() - t0
    n_all = count * cores
    t0 = time.perf_counter()
    seeds, _, cov = pool.max_coverage(count, min(k, el.n))
    t_greedy = time.perf_counter() - t0
    t0 = time.perf_counter()
    pool.coverage(0, count, seeds)
    t_stare = time.perf_counter() - t0
    return {"value": n_all / t_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": (f"sampling phase of the step-0 solve's stream: sets [{count}, {count + n_all}) over "
                       f"{used} threads by sample range ({t_all:.1f} s); one thread: sets [0, {count}) "
                       f"({t_one:.1f} s); Max-Coverage k={min(k, el.n)} and the stare count over those "
                       f"{count} sets"),
            "single_thread": {"value": count / t_one, "unit": UNIT, "cores": 1},
            "phases_s": {"sample_1_thread": t_one, "sample_all_cores": t_all, "greedy_1_thread": t_greedy,
                         "stare_1_thread": t_stare, "graph_build_1_thread": t_graph},
            "sets_one_thread": count, "sets_all_cores": n_all}


def run_reference(args):
    """The oracle on the host cores, as it stands: per step, the sampling phase of
    a solve's stream (Philox seed = step index + 1) for a bounded number of sets,
    over all cores by sample range."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    name = args.workload
    el, weighting, algo, model, k, eps = make_graph_inputs(name)
    import oracle
    oracle.build()
    og = oracle.Graph(el.n, el.src, el.dst, weighting, None, 1)
    cores = os.cpu_count() or 1
    per_step = args.ref_sets if args.ref_sets > 0 else 64 * cores
    times, used = [], 1
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        used, _, _ = oracle.sample_threads(og, model, 1 + s, 0, 0, per_step, cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total_t = sum(times)
    value = per_step * args.steps / total_t
    sample = (f"first {per_step} RR sets of each step's solve stream (Philox seed = step index + 1), "
              f"sampling phase only, {used} host threads by sample range")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": name, "n": el.n, "m": el.m, "k": k, "eps": eps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_queries(nq, graphs_n, seed=7):
    """c5 query mix: graph and model 50/50, k in {1,10,100,1000}, eps in {0.05,0.1,0.2},
    delta = 1/n, seed = query index, every other query targeted (Zipf benefits)."""
    import inputs
    u = inputs.uniforms(6 * nq, seed).reshape(nq, 6)
    qs = []
    for i in range(nq):
        g = int(u[i, 0] * 2)
        qs.append({"graph": g, "model": int(u[i, 1] * 2), "k": [1, 10, 100, 1000][int(u[i, 2] * 4)],
                   "eps": [0.05, 0.1, 0.2][int(u[i, 3] * 3)], "delta": 1.0 / graphs_n[g], "seed": i,
                   "targeted": i % 2 == 1})
    return qs


def run_serving(args):
    """The serving mix alone (bench.py --serving), as one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_07990_gb300 as P
    torch.cuda.set_device(0)
    P.ssa_set_greedy_mode(args.greedy_mode)
    line = serving(P, args.queries, args.slots)
    line["greedy_mode"] = args.greedy_mode
    line.update({"metric": "serving queries/s and p50/p99 latency", "unit": "queries/s",
                 "value": line["server"]["queries_per_s"], "higher_is_better": True, "n_gpus": 1,
                 "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def serving(P, nq, slots):
    """Poisson stream of mixed queries against two resident graphs: the serving
    loop (continuous admission, concurrent slots, CUDA-graph rounds) against
    sequential solves through the same library."""
    import inputs
    els = [inputs.rmat(20, 1 << 24, seed=1), inputs.rmat(23, 1 << 27, seed=1)]
    gs = [P.ssa_load_graph(e.n, e.src, e.dst, None, P.SSA_W_WC) for e in els]
    ws = [inputs.zipf_benefit(e.n, 1.2, seed=100 + i) for i, e in enumerate(els)]
    qs = serving_queries(nq, [e.n for e in els])

    def solve_seq(algo):
        solvers = [P.Solver(g) for g in gs]
        out, svc = [], []
        for q in qs:
            b = ws[q["graph"]] if q["targeted"] else None
            t0 = time.perf_counter()
            r = solvers[q["graph"]].solve(algo, q["model"], q["k"], q["eps"], q["delta"], q["seed"], benefit=b)
            svc.append(time.perf_counter() - t0)
            out.append(r)
        for s_ in solvers:
            s_.free()
        return out, np.array(svc)

    # warm-up: first solves pay for workspace allocation
    for g, e in zip(gs, els):
        P.ssa_solve(g, 1, 0, 10, 0.1, 1.0 / e.n, 12345)
    seq_d, svc_d = solve_seq(P.SSA_ALGO_DSSA)
    seq_s, svc_s = solve_seq(P.SSA_ALGO_SSA)
    # Poisson arrivals at 0.8 of the sequential D-SSA capacity
    rate = 0.8 / float(svc_d.mean())
    arr = np.cumsum(-np.log1p(-inputs.uniforms(len(qs), 4242)) / rate)

    def fifo(svc):
        fin, lat = 0.0, []
        for a, s_ in zip(arr, svc):
            fin = max(a, fin) + s_
            lat.append(fin - a)
        lat = np.array(lat)
        return {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                "queries_per_s": len(qs) / fin, "saturated_queries_per_s": len(qs) / float(svc.sum())}

    srv = P.Server(gs, slots=slots)
    t0 = time.perf_counter()
    tickets = []
    for q, a in zip(qs, arr):
        delay = a - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        b = ws[q["graph"]] if q["targeted"] else None
        tickets.append(srv.submit(q["graph"], P.SSA_ALGO_DSSA, q["model"], q["k"], q["eps"], q["delta"],
                                  q["seed"], benefit=b))
    live = [srv.wait(t) for t in tickets]
    t_live = time.perf_counter() - t0
    lat = np.array([r.latency_s for r in live])
    same = sum(int(np.array_equal(x.seeds, y.seeds) and x.trace == y.trace) for x, y in zip(seq_d, live))
    # saturated: everything at once
    t1 = time.perf_counter()
    tk = [srv.submit(q["graph"], P.SSA_ALGO_DSSA, q["model"], q["k"], q["eps"], q["delta"], q["seed"],
                     benefit=ws[q["graph"]] if q["targeted"] else None) for q in qs]
    sat = [srv.wait(t) for t in tk]
    t_sat = time.perf_counter() - t1
    srv.close()
    line = {"config": {"workload": "Poisson mix: R-MAT 2^20/2^24 and 2^23/2^27 (WC weights), IC/LT, "
                                   "k in {1,10,100,1000}, eps in {0.05,0.1,0.2}, half targeted (Zipf 1.2)",
                       "queries": len(qs), "arrival_rate_per_s": rate, "slots": slots},
            "server": {"p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                       "queries_per_s": len(qs) / t_live, "saturated_queries_per_s": len(qs) / t_sat,
                       "answers_equal_to_sequential": same, "saturated_answers": len(sat)},
            "sequential_dssa": fifo(svc_d), "sequential_plain_ssa": fifo(svc_s),
            "mean_service_ms": {"dssa": 1e3 * float(svc_d.mean()), "ssa": 1e3 * float(svc_s.mean())}}
    for g in gs:
        g.free()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--extra-steps", type=int, default=5, help="steps of the D-SSA trivalency workload (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="one-thread sampling time of the CPU baseline")
    ap.add_argument("--ref-sets", type=int, default=0, help="RR sets per reference step (0: 64 per host core)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--sample-only", type=int, default=0,
                    help="profiling case: only sample this many RR sets of the workload into a pool")
    ap.add_argument("--then-greedy", type=int, default=0,
                    help="with --sample-only: also index the pool and run greedy Max-Coverage for this k")
    ap.add_argument("--tune", default="",
                    help="with --sample-only: IC sampler hand-overs MID_CAP,HEAVY_GROUPS[,GLOBAL_BITMAP_TIER] "
                         "(ssa_set_tuning, ssa_set_warp_tier)")
    ap.add_argument("--serving", action="store_true", help="the Poisson serving mix instead of the solve bench")
    ap.add_argument("--queries", type=int, default=2000, help="queries of --serving")
    ap.add_argument("--serving-queries", type=int, default=120,
                    help="queries of the serving mix measured after the solve bench (0: skip)")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--greedy-mode", type=int, default=0,
                    help="greedy launch shape (ssa_set_greedy_mode): 0 by pool size, 1 grid, 2 cluster")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serving:
        return run_serving(args)

    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1605_07990_gb300 as P

    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count
    name = args.workload
    el, weighting, algo, model, k, eps = make_graph_inputs(name)
    delta = 1.0 / el.n
    g = P.ssa_load_graph(el.n, el.src, el.dst, None, weighting, 1)
    og_thread = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.sample_only:
        og_thread = OracleGraph(el, weighting)
        og_thread.start()
    if args.sample_only:
        if args.tune:
            t = [int(x) for x in args.tune.split(",")]
            P.ssa_set_tuning(g, t[0], t[1])
            if len(t) > 2:
                P.ssa_set_warp_tier(g, t[2])
        t0 = time.perf_counter()
        pool = P.Pool(g, model, seed=1, stream=0).grow(args.sample_only)
        torch.cuda.synchronize()
        out = {"sample_only": args.sample_only, "pool": pool.info(), "seconds": time.perf_counter() - t0,
               "tune": args.tune}
        if args.then_greedy:
            _, gains, cov = pool.max_coverage(args.sample_only, args.then_greedy)
            out["greedy"] = {"k": args.then_greedy, "cov": int(cov)}
        print(json.dumps(out))
        pool.free()
        g.free()
        return 0
    stream = torch.cuda.current_stream()
    solver = P.Solver(g, stream=stream.cuda_stream)

    def seed_of(step):
        return replica_seed(rank, step)

    if world > 1:
        dist.barrier()
    try:
        gpu_id = props.uuid
        gpu_id = f"GPU-{gpu_id}" if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    except Exception:
        gpu_id = local
    # warm-up outside the clock sampler, then the timed steps with it
    run_solves(P, solver, name, 0, args.warmup, seed_of, stream, torch)
    if world > 1:
        dist.barrier()
    clk = Clocks(gpu_id)
    clk.start()
    results, ms = run_solves(P, solver, name, args.steps, 0, seed_of, stream, torch)
    clocks = clk.stop()
    clock_mhz = clocks.get("sm_mhz") or 2070.0
    rr = sum(r.n_rr for r in results)
    ev = sum(r.edge_visits for r in results)
    nv = sum(r.node_visits for r in results)
    if world > 1:
        ms_max, (rr_all, ev_all, nv_all) = reduce_over_ranks(ms, (rr, ev, nv), "cuda")
    else:
        ms_max, rr_all, ev_all, nv_all = ms, float(rr), float(ev), float(nv)
    summ = summarise(P, name, results, ms, sm_count, clock_mhz)
    value = rr_all / (ms_max / 1000.0)
    cfg = {"workload": name, "n": el.n, "m": el.m, "algo": "D-SSA" if algo else "SSA",
           "model": "LT" if model else "IC", "weights": WEIGHTS[weighting], "k": k, "eps": eps, "delta": "1/n",
           "parallelism": f"replicas{world}",
           "l2": f"inputs larger than L2 (CSR {P.ssa_graph_info(g)[2] / 1e9:.2f} GB; RR pool several GB per solve)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": cfg,
            "edge_visits_per_s": ev_all / (ms_max / 1000.0), "node_visits_per_s": nv_all / (ms_max / 1000.0)}
    for key in ("philox_draws_per_s", "rr_sets_per_solve", "rr_sets_stored_per_solve",
                "rr_sets_hit_tested_per_solve", "rounds", "kernel_ms", "gpu_launches"):
        line[key] = summ[key]
    line["clocks"] = clocks
    line["roofline"] = summ["roofline"]

    if og_thread is not None:
        og_thread.join()  # host memory traffic of the oracle's build stays out of the e2e leg
    # end to end through the C ABI: pinned host edges -> graph upload + device CSR build -> solve -> seeds to host
    src_h = torch.from_numpy(el.src).pin_memory()
    dst_h = torch.from_numpy(el.dst).pin_memory()
    src_np, dst_np = src_h.numpy(), dst_h.numpy()
    torch.cuda.synchronize()
    rr_e2e, t_load, t_solve = 0, 0.0, 0.0
    t0 = time.perf_counter()
    for s in range(args.e2e_steps):
        ta = time.perf_counter()
        g2 = P.ssa_load_graph(el.n, src_np, dst_np, None, weighting, 1)
        tb = time.perf_counter()
        # the timed steps' own seeds, so both legs draw the same RR sets
        r = P.ssa_solve(g2, algo, model, k, eps, delta, seed_of(s))
        tc = time.perf_counter()
        rr_e2e += r.n_rr
        g2.free()
        t_load += tb - ta
        t_solve += tc - tb
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    if args.e2e_steps > 0:
        line["e2e"] = {"value": rr_e2e / te, "unit": UNIT, "h2d_bytes_per_step": int(el.m * 8),
                       "d2h_bytes_per_step": int(k * 4 + 64), "steps": args.e2e_steps,
                       "includes": "graph upload + device CSR build (and, under weighted cascade, the gap-power "
                                   "table) + solve (the first solve on a new graph handle picks the sampler tiers) "
                                   "+ seeds to host",
                       "load_s_per_step": t_load / args.e2e_steps, "solve_s_per_step": t_solve / args.e2e_steps,
                       "seeds": "the first e2e steps use the timed steps' Philox seeds"}

    if args.extra_steps > 0 and name != EXTRA:
        el2, w2, _, _, _, _ = make_graph_inputs(EXTRA)
        g3 = P.ssa_load_graph(el2.n, el2.src, el2.dst, None, w2, 1)
        solver3 = P.Solver(g3, stream=stream.cuda_stream)
        res3, ms3 = run_solves(P, solver3, EXTRA, args.extra_steps, 2, seed_of, stream, torch)
        ex = summarise(P, EXTRA, res3, ms3, sm_count, clock_mhz)
        ex["config"] = {"n": el2.n, "m": el2.m, "algo": "D-SSA", "model": "IC", "weights": "trivalency", "k": 100,
                        "eps": 0.1, "delta": "1/n", "l2": "CSR 137 MB: mostly L2-resident"}
        ex["steps"] = args.extra_steps
        line["extra"] = {EXTRA: ex}
        solver3.free()
        g3.free()

    if args.serving_queries > 0 and world == 1:
        line["serving"] = serving(P, args.serving_queries, args.slots)
    if og_thread is not None:
        if og_thread.g is None:
            line["cpu_baseline"] = {"unavailable": f"oracle graph build failed: {og_thread.error}"}
        else:
            line["cpu_baseline"] = cpu_baseline(og_thread.g, og_thread.seconds, el, model, k, seed_of(0),
                                                args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.free()
    g.free()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
