// Serving loop: continuous admission of influence-maximisation queries
// against graphs kept resident on the device (ssa_server_* in include/ssa.h).
//
// A fixed set of worker slots, each with its own CUDA stream and per-graph
// solver workspaces, drains one FIFO of requests.  The head request is
// admitted as soon as a slot is free and its estimated RR-pool footprint fits
// the server's byte budget (footprints are learned per (graph, model, k) from
// finished requests).  Admitted requests run concurrently on their slots'
// streams, so their sampling, index, greedy and stare kernels overlap on the
// GPU while later arrivals wait for a slot or for memory.  Every request's
// randomness is keyed by its own seed, so its answer does not depend on what
// else is in flight.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ssa.h"
#include "kernels.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  int graph = 0;
  ssa_params p{};
  std::vector<uint32_t> benefit;
  std::vector<int32_t> seeds;
  std::vector<ssa_round> trace;
  ssa_result res{};
  ssa_status status = SSA_OK;
  bool done = false;
  double t_submit = 0, t_start = 0, t_done = 0;
  int64_t reserved = 0;
};

ssa_status fail_msg(ssa_status s, const char* msg) {
  ssa::set_last_error(msg);
  return s;
}

}  // namespace

struct ssa_server {
  int device = 0;
  std::vector<const ssa_graph*> graphs;
  int64_t budget = 0;
  int64_t in_use = 0;
  int active = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  std::map<std::tuple<int, int, int>, int64_t> footprint;  // (graph, model, k bucket) -> bytes
  std::vector<std::thread> workers;
  int64_t submitted = 0, completed = 0, failed = 0;
  std::vector<double> latencies;  // seconds, completed requests

  int64_t estimate(const Request& r) {
    const int kb = r.p.k <= 1 ? 0 : r.p.k <= 10 ? 1 : r.p.k <= 100 ? 2 : 3;
    auto it = footprint.find({r.graph, (int)r.p.model, kb});
    return it == footprint.end() ? (int64_t)256 << 20 : it->second;
  }
  void learn(const Request& r, int64_t bytes) {
    const int kb = r.p.k <= 1 ? 0 : r.p.k <= 10 ? 1 : r.p.k <= 100 ? 2 : 3;
    auto key = std::make_tuple(r.graph, (int)r.p.model, kb);
    auto it = footprint.find(key);
    // keep the largest footprint seen, with a margin: admission must not starve memory
    const int64_t b = bytes + bytes / 4;
    if (it == footprint.end() || it->second < b) footprint[key] = b;
  }

  void worker_main() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<ssa_solver*> solvers(graphs.size(), nullptr);
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lock(mu);
        cv_work.wait(lock, [&] {
          if (stop) return true;
          if (pending.empty()) return false;
          const int64_t need = estimate(*pending.front());
          // admit when it fits, or when nothing else runs (progress is guaranteed)
          return active == 0 || in_use + need <= budget;
        });
        if (stop && pending.empty()) break;
        if (stop) {
          // shutting down: cancel what never started
          while (!pending.empty()) {
            Request* q = pending.front();
            pending.pop_front();
            q->status = SSA_E_CANCELLED;
            q->done = true;
            q->t_done = now_s();
          }
          cv_done.notify_all();
          break;
        }
        r = pending.front();
        pending.pop_front();
        r->reserved = estimate(*r);
        // hard cap: everything the others have not reserved
        r->p.pool_bytes_cap = std::max<int64_t>(budget - in_use, r->reserved);
        in_use += r->reserved;
        active += 1;
        r->t_start = now_s();
      }
      ssa_status s = SSA_OK;
      if (!solvers[(size_t)r->graph]) {
        s = ssa_solver_create(graphs[(size_t)r->graph], st, 0, &solvers[(size_t)r->graph]);
        // each round's index, greedy and stare as one CUDA graph, reused by later requests;
        // the greedy in one thread-block cluster, so concurrent requests keep the other SMs
        if (s == SSA_OK) s = ssa_solver_set_graphs(solvers[(size_t)r->graph], 1);
        if (s == SSA_OK) s = ssa_solver_set_shared(solvers[(size_t)r->graph], 1);
      }
      if (s == SSA_OK) {
        r->seeds.assign((size_t)r->p.k, -1);
        r->trace.assign(64, ssa_round{});
        std::memset(&r->res, 0, sizeof(r->res));
        r->res.seeds = r->seeds.data();
        r->res.trace = r->trace.data();
        r->res.trace_cap = 64;
        if (!r->benefit.empty()) r->p.benefit = r->benefit.data();
        s = ssa_solver_solve(solvers[(size_t)r->graph], &r->p, &r->res);
      }
      {
        std::lock_guard<std::mutex> lock(mu);
        r->status = s;
        r->done = true;
        r->t_done = now_s();
        in_use -= r->reserved;
        active -= 1;
        if (s == SSA_OK) {
          completed += 1;
          latencies.push_back(r->t_done - r->t_submit);
          learn(*r, r->res.pool_entries * 16 + r->res.n_rr * 16);
        } else {
          failed += 1;
        }
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    for (auto* s : solvers)
      if (s) ssa_solver_free(s);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
};

extern "C" {

ssa_status ssa_server_create(const ssa_graph* const* graphs, int32_t n_graphs, int32_t slots, int64_t pool_bytes,
                             ssa_server** out) {
  if (!out || !graphs || n_graphs < 1 || slots < 1 || slots > 64)
    return fail_msg(SSA_E_ARG, "ssa_server_create: need graphs, 1 <= slots <= 64");
  for (int i = 0; i < n_graphs; ++i)
    if (!graphs[i]) return fail_msg(SSA_E_ARG, "ssa_server_create: null graph");
  ssa_server* s = new ssa_server();
  cudaGetDevice(&s->device);
  s->graphs.assign(graphs, graphs + n_graphs);
  if (pool_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    pool_bytes = (int64_t)((double)fr * 0.6);
  }
  s->budget = pool_bytes;
  for (int i = 0; i < slots; ++i) s->workers.emplace_back([s] { s->worker_main(); });
  *out = s;
  return SSA_OK;
}

ssa_status ssa_server_submit(ssa_server* s, int32_t graph, const ssa_params* p, uint64_t* ticket) {
  if (!s || !p || !ticket) return fail_msg(SSA_E_ARG, "ssa_server_submit: null argument");
  if (graph < 0 || graph >= (int)s->graphs.size()) return fail_msg(SSA_E_ARG, "ssa_server_submit: bad graph index");
  int64_t n = 0;
  ssa_graph_info(s->graphs[(size_t)graph], &n, nullptr, nullptr);
  if (p->k < 1 || p->k > n) return fail_msg(SSA_E_ARG, "ssa_server_submit: k outside [1, n]");
  auto r = std::make_unique<Request>();
  r->graph = graph;
  r->p = *p;
  if (p->benefit) r->benefit.assign(p->benefit, p->benefit + n);
  r->p.benefit = nullptr;
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return fail_msg(SSA_E_CANCELLED, "ssa_server_submit: server is shutting down");
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->pending.push_back(r.get());
    s->all[r->ticket] = std::move(r);
    s->submitted += 1;
  }
  s->cv_work.notify_one();
  return SSA_OK;
}

static ssa_status take_result(ssa_server* s, std::unique_lock<std::mutex>& lock, uint64_t ticket, int32_t* seeds,
                              ssa_result* out, double* latency_s) {
  auto it = s->all.find(ticket);
  Request* r = it->second.get();
  const ssa_status st = r->status;
  if (st == SSA_OK) {
    if (out) {
      ssa_round* tr = out->trace;
      const int32_t cap = out->trace_cap;
      *out = r->res;
      out->seeds = seeds;
      out->trace = tr;
      out->trace_cap = cap;
      if (tr && cap > 0) std::memcpy(tr, r->trace.data(), sizeof(ssa_round) * (size_t)std::min(cap, 64));
    }
    if (seeds) std::memcpy(seeds, r->seeds.data(), sizeof(int32_t) * r->seeds.size());
  }
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  s->all.erase(it);
  (void)lock;
  if (st != SSA_OK) return fail_msg(st, "ssa_server: request failed");
  return SSA_OK;
}

ssa_status ssa_server_poll(ssa_server* s, uint64_t ticket, int32_t* seeds, ssa_result* out, double* latency_s) {
  if (!s) return fail_msg(SSA_E_ARG, "ssa_server_poll: null server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail_msg(SSA_E_ARG, "ssa_server_poll: unknown ticket");
  if (!it->second->done) return SSA_E_NOT_READY;
  return take_result(s, lock, ticket, seeds, out, latency_s);
}

ssa_status ssa_server_wait(ssa_server* s, uint64_t ticket, double timeout_s, int32_t* seeds, ssa_result* out,
                           double* latency_s) {
  if (!s) return fail_msg(SSA_E_ARG, "ssa_server_wait: null server");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail_msg(SSA_E_ARG, "ssa_server_wait: unknown ticket");
  Request* r = it->second.get();
  const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [&] { return r->done; });
  if (!ok) return fail_msg(SSA_E_TIMEOUT, "ssa_server_wait: not done in time");
  return take_result(s, lock, ticket, seeds, out, latency_s);
}

ssa_status ssa_server_stats(ssa_server* s, ssa_serve_stats* out) {
  if (!s || !out) return fail_msg(SSA_E_ARG, "ssa_server_stats: null argument");
  std::lock_guard<std::mutex> lock(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->active = s->active;
  out->pending = (int64_t)s->pending.size();
  out->bytes_budget = s->budget;
  out->bytes_in_use = s->in_use;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  auto q = [&](double f) { return l.empty() ? 0.0 : 1e3 * l[(size_t)std::min<double>(l.size() - 1, f * l.size())]; };
  out->p50_ms = q(0.50);
  out->p99_ms = q(0.99);
  return SSA_OK;
}

ssa_status ssa_server_destroy(ssa_server* s) {
  if (!s) return SSA_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
  return SSA_OK;
}

}  // extern "C"
