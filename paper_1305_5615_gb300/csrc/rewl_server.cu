// rewl_server.cu -- the served form of REWL: density-of-states requests of
// different models and lattice sizes arrive at any time, are admitted while
// request slots and the device-memory budget allow, and run together.
//
// Running requests are grouped by shape (model, L): the walkers of one group
// all take about the same time per block, so a group advances in rounds --
// (a shape whose round lasts milliseconds gives each request a group of its
// own: there a round is latency-bound per walker, and a fused round would make
// every request wait for the slowest walker of all of them) --
// one fused sweep launch over every walker of every request of the group,
// then one launch each for the exchanges, the clocks and the due flatness
// checks of all its requests.  The device decides every phase boundary: the
// clocks, the flatness checks, the merges and the done flags live in device
// memory and the kernels of a finished window or request do nothing, so
// several rounds run back to back without the host.  A group's k rounds and
// the small report read back after them are captured once as a CUDA graph
// and replayed (captured again when the group's table or sweep form changes);
// k adapts so that one replay lasts a few milliseconds.  Each group has a
// CUDA stream of its own and its replays are issued as soon as the previous
// one has been read, so groups of different sizes run side by side on the
// GPU at their own pace (a 12 x 12 glass is not held back by a 32 x 32 Potts
// lattice).  Requests are admitted while request slots, the memory budget and
// the target of active walkers (walkers of windows not done) allow, so that
// finishing windows make room for new requests.  Requests that finish are
// retired when their group's replay has been read: their joined ln g is read
// back and their memory goes to the queue.  Every request keeps its own seed,
// schedule and state, so its result is bit-identical to the one it gets alone
// (rewl_create + rewl_step).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rewl.h"
#include "rewl_ctx.h"
#include "rewl_kernels.h"
#include "rewl_layout.h"

using namespace rewl;
using Clock = std::chrono::steady_clock;

namespace {

rewl_status sfail(rewl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  rewl_set_last_error(buf);
  return s;
}

#define SCUDA(expr)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (expr);                                                                         \
    if (e_ != cudaSuccess) return sfail(REWL_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));        \
  } while (0)

struct Request {
  uint64_t id = 0;
  int state = REWL_REQ_QUEUED;
  rewl_status error = REWL_OK;
  rewl_model model{};
  rewl_lattice lattice{};
  std::vector<int8_t> couplings;
  bool has_couplings = false;
  int32_t windows = 0, walkers_per_window = 0;
  double overlap = 0, flatness = 0, lnf_final = 0;
  uint64_t seed = 0;
  int64_t bytes = 0;
  Clock::time_point t_submit, t_admit, t_done;
  rewl_ctx* ctx = nullptr;
  int group = -1, slot = -1;
  int n_done = 0;
  int64_t sweeps = 0, attempts = 0;
  int64_t active_walkers = 0;  // walkers of windows not done (from the last report)
  std::vector<double> lng;
  int32_t n_bins = 0, e_min = 0, e_step = 0;
};

// Device bytes a request may use: its per-walker arrays with the widest
// window its energy range allows, plus per-window tables.
int64_t request_bytes(const Request& r) {
  const int L = r.lattice.Lx, dim = r.lattice.dim;
  const int64_t rows = dim == 3 ? (int64_t)L * L : L, N = rows * L;
  const bool potts = r.model.kind == REWL_POTTS;
  const int Wr = potts ? (L + 7) / 8 : (L + 31) / 32, Wr1 = (L + 31) / 32;
  const int64_t lat_words = rows * Wr;
  const int64_t B = potts ? 2LL * N + 1 : (int64_t)dim * N / 2 + 1;  // the widest grid the model can have
  int64_t w = B;
  if (r.windows > 1)
    w = std::min<int64_t>(B, (int64_t)std::ceil((double)B / (1.0 + (double)(r.windows - 1) * (1.0 - r.overlap))));
  w = std::min<int64_t>(B, 2 * w);  // first and last windows reach on to the ends of a +-J grid
  const int64_t nW = (int64_t)r.windows * r.walkers_per_window;
  return nW * (lat_words * 4 + 4 + w * 12 + 3 * 8 + 3 * 4 + 8) + (int64_t)r.windows * 64 + lat_words * 4 +
         (int64_t)dim * rows * Wr1 * 4 + 4096;
}

// Running requests of one shape (model, L) and the device tables of their rounds.
// `slots` is the host copy of the slot table; it is staged through pinned memory
// and uploaded only when a round is issued, i.e. while no round of the group is
// in flight, so the staging buffers are never rewritten under a pending copy.
struct Group {
  int model = 0, L = 0;
  bool priv = false;                // serves one request at a time (a shape with long rounds)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;
  bool in_flight = false;
  std::vector<uint64_t> slot_req;   // request id per slot, 0 = free
  std::vector<uint64_t> launched;   // request id per slot in the round in flight
  std::vector<BatchSlot> slots;     // slot table
  int cap = 0;                      // slots the device tables hold
  BatchSlot* h_stage = nullptr;     // pinned [cap]
  BatchSlot* d_slots = nullptr;     // [cap]
  SlotReport* h_rep = nullptr;      // pinned [cap]
  SlotReport* d_rep = nullptr;      // [cap]
  BatchWalker* h_list = nullptr;    // pinned [list_cap]: every walker, then (from n_list) every quad
  BatchWalker* d_list = nullptr;    // [list_cap]
  int list_cap = 0, n_list = 0, n_quad = 0, hi = 0;  // hi: slots [0, hi) in the round
  size_t smem = 0, smem_quad = 0;
  int max_pairs = 0, max_m = 1, max_h = 1;
  bool dirty = true;
  // the captured replay: k rounds and the report, for one table and one sweep form
  cudaGraphExec_t exec = nullptr;
  int exec_form = -1, exec_k = 0;
  int k = 1;                        // rounds per replay (adapted to about kReplayMs)
  Clock::time_point t_launch;

  ~Group() {
    if (stream) cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(d_slots);
    cudaFree(d_rep);
    cudaFree(d_list);
    if (h_stage) cudaFreeHost(h_stage);
    if (h_rep) cudaFreeHost(h_rep);
    if (h_list) cudaFreeHost(h_list);
    if (ev) cudaEventDestroy(ev);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  int running() const {
    int n = 0;
    for (uint64_t id : slot_req) n += id != 0;
    return n;
  }
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

constexpr double kReplayMs = 4.0;  // target duration of one replay of a shared group's rounds
constexpr double kPrivateReplayMs = 32.0;  // ... of a private group's (its request runs for seconds)
constexpr double kPrivateRoundMs = 2.0;  // estimated round length from which requests get a group each
constexpr int kMaxRoundsPerReplay = 16;

struct rewl_server {
  std::mutex mu;
  rewl_params params{};
  int64_t budget = 0, in_use = 0;
  int max_running = 0, n_running = 0;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<std::unique_ptr<Group>> groups;
  int64_t rounds = 0, attempts = 0;
  int finished = 0, failed = 0;
  int n_sm = 152;
  int64_t walker_target = 0;  // admission stops while this many walkers are active (0 = no limit)

  int64_t active_walkers() const {
    int64_t n = 0;
    for (const auto& gp : groups)
      for (size_t s = 0; s < gp->slots.size(); ++s)
        if (gp->slot_req[s]) n += reqs.at(gp->slot_req[s]).active_walkers;
    return n;
  }

  ~rewl_server() {
    for (auto& g : groups)
      if (g->stream) cudaStreamSynchronize(g->stream);
    for (auto& kv : reqs)
      if (kv.second.ctx) rewl_destroy(kv.second.ctx);
    groups.clear();
  }

  // The group a new request of shape (model, L) joins: the shape's shared group, or -- for
  // shapes whose rounds are long (priv) -- an idle private group of the shape, else a new one.
  rewl_status group_for(int model, int L, bool priv, int* out) {
    for (size_t i = 0; i < groups.size(); ++i) {
      const Group& g = *groups[i];
      if (g.model != model || g.L != L || g.priv != priv) continue;
      if (priv && (g.running() > 0 || g.in_flight)) continue;
      *out = (int)i;
      return REWL_OK;
    }
    auto g = std::make_unique<Group>();
    g->model = model;
    g->L = L;
    g->priv = priv;
    if (params.stream) {
      g->stream = (cudaStream_t)params.stream;
    } else {
      SCUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
      g->own_stream = true;
    }
    SCUDA(cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming));
    groups.push_back(std::move(g));
    *out = (int)groups.size() - 1;
    return REWL_OK;
  }

  // A free slot of group g (host tables only; the device tables follow at the next round).
  int take_slot(Group& g) {
    for (size_t i = 0; i < g.slot_req.size(); ++i)
      if (!g.slot_req[i]) return (int)i;
    g.slot_req.push_back(0);
    g.launched.push_back(0);
    g.slots.push_back(BatchSlot{});
    return (int)g.slot_req.size() - 1;
  }

  // Admission: first-come first-served while a slot, the memory budget and the
  // target of active walkers allow (the first request is always admitted).
  rewl_status admit() {
    int64_t active = active_walkers();
    while (!queue.empty()) {
      const uint64_t id = queue.front();
      Request& r = reqs[id];
      if (n_running >= max_running || in_use + r.bytes > budget) break;  // head of queue waits
      if (walker_target > 0 && n_running > 0 && active >= walker_target) break;
      queue.pop_front();
      rewl_params p = params;
      p.stream = params.stream;  // NULL: the request gets a stream of its own for its set-up
      p.lanes_per_walker = 32;
      p.walkers_per_block = 1;
      p.mode = REWL_MODE_PLAIN;
      p.profile = 0;
      p.prefetch_draws = 0;  // the batched kernels draw in-kernel
      rewl_handle h = nullptr;
      const rewl_status st = rewl_create(&h, &r.model, &r.lattice, r.has_couplings ? r.couplings.data() : nullptr,
                                         r.windows, r.overlap, r.walkers_per_window, r.flatness, r.lnf_final, r.seed,
                                         &p);
      if (st != REWL_OK) {
        r.state = REWL_REQ_FAILED;
        r.error = st;
        r.t_done = Clock::now();
        ++failed;
        continue;
      }
      // Requests of one shape share a group (one fused launch per phase for all of them) while a
      // round is short, i.e. launch-bound; a shape whose round lasts milliseconds (one block of
      // N x sweeps_per_exchange trials of a walker, about 75 ns each) is latency-bound per walker,
      // and its requests get a group each, so that no request waits for another's slowest walker.
      const double round_ms = 75e-6 * (double)h->P.N * (double)h->params.sweeps_per_exchange;
      int gi = -1;
      const rewl_status gs = group_for(r.model.kind, r.lattice.Lx, round_ms >= kPrivateRoundMs, &gi);
      if (gs != REWL_OK) {
        rewl_destroy(h);
        return gs;
      }
      Group& g = *groups[gi];
      const int s = take_slot(g);
      r.ctx = h;
      r.group = gi;
      r.slot = s;
      r.state = REWL_REQ_RUNNING;
      r.t_admit = Clock::now();
      in_use += r.bytes;
      ++n_running;
      r.active_walkers = h->P.n_walkers;
      active += r.active_walkers;
      g.slot_req[s] = id;
      BatchSlot& b = g.slots[s];
      b.P = h->P;
      b.S = h->S;
      b.spe = (uint32_t)h->params.sweeps_per_exchange;
      b.spf = (uint32_t)h->params.sweeps_per_flat_check;
      b.n_att = b.spe * (uint32_t)h->P.N;
      b.active = 1;
      g.dirty = true;
    }
    return REWL_OK;
  }

  // Uploads the group's slot table and walker list (before a launch, nothing in flight).
  rewl_status rebuild(Group& g) {
    const int need = (int)g.slots.size();
    if (need > g.cap) {
      const int cap = std::max(need, 2 * g.cap);
      BatchSlot *hs = nullptr, *ds = nullptr;
      SlotReport *hr = nullptr, *dr = nullptr;
      if (cudaMallocHost(&hs, sizeof(BatchSlot) * cap) != cudaSuccess ||
          cudaMallocHost(&hr, sizeof(SlotReport) * cap) != cudaSuccess ||
          cudaMalloc(&ds, sizeof(BatchSlot) * cap) != cudaSuccess ||
          cudaMalloc(&dr, sizeof(SlotReport) * cap) != cudaSuccess) {
        if (hs) cudaFreeHost(hs);
        if (hr) cudaFreeHost(hr);
        cudaFree(ds);
        cudaFree(dr);
        return sfail(REWL_ENOMEM, "group tables of %d slots", cap);
      }
      if (g.h_stage) cudaFreeHost(g.h_stage);
      if (g.h_rep) cudaFreeHost(g.h_rep);
      cudaFree(g.d_slots);
      cudaFree(g.d_rep);
      g.h_stage = hs;
      g.h_rep = hr;
      g.d_slots = ds;
      g.d_rep = dr;
      g.cap = cap;
    }
    int n = 0, nq = 0, hi = 0;
    g.max_pairs = 0;
    g.max_m = 1;
    g.max_h = 1;
    g.smem = 0;
    g.smem_quad = 0;
    for (int s = 0; s < need; ++s) {
      g.h_stage[s] = g.slots[s];
      if (!g.slot_req[s]) continue;
      const Problem& P = g.slots[s].P;
      n += P.n_walkers;
      nq += (P.n_walkers + 3) / 4;
      hi = s + 1;
      g.smem = std::max(g.smem, sweep_smem_bytes(P, 1, 32, kSweepChain));
      g.smem_quad = std::max(g.smem_quad, sweep_smem_bytes(P, 4, 8, kSweepChain));
      g.max_pairs = std::max(g.max_pairs, P.h / 2);
      g.max_m = std::max(g.max_m, P.m);
      g.max_h = std::max(g.max_h, P.h);
    }
    g.hi = hi;
    if (n + nq > g.list_cap) {
      const int cap = std::max(n + nq, 2 * g.list_cap);
      BatchWalker *hl = nullptr, *dl = nullptr;
      if (cudaMallocHost(&hl, sizeof(BatchWalker) * cap) != cudaSuccess ||
          cudaMalloc(&dl, sizeof(BatchWalker) * cap) != cudaSuccess) {
        if (hl) cudaFreeHost(hl);
        cudaFree(dl);
        return sfail(REWL_ENOMEM, "walker list of %d entries", cap);
      }
      if (g.h_list) cudaFreeHost(g.h_list);
      cudaFree(g.d_list);
      g.h_list = hl;
      g.d_list = dl;
      g.list_cap = cap;
    }
    int k = 0;
    for (int s = 0; s < hi; ++s) {
      if (!g.slot_req[s]) continue;
      for (int W = 0; W < g.slots[s].P.n_walkers; ++W) g.h_list[k++] = BatchWalker{s, W};
    }
    for (int s = 0; s < hi; ++s) {
      if (!g.slot_req[s]) continue;
      for (int W = 0; W < g.slots[s].P.n_walkers; W += 4) g.h_list[k++] = BatchWalker{s, W};
    }
    g.n_list = n;
    g.n_quad = nq;
    if (hi) SCUDA(cudaMemcpyAsync(g.d_slots, g.h_stage, sizeof(BatchSlot) * hi, cudaMemcpyHostToDevice, g.stream));
    if (n + nq)
      SCUDA(cudaMemcpyAsync(g.d_list, g.h_list, sizeof(BatchWalker) * (n + nq), cudaMemcpyHostToDevice, g.stream));
    g.dirty = false;
    if (g.exec) {  // the replay read the old tables' sizes: capture again
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    return REWL_OK;
  }

  // Captures g.k rounds of the group in the given sweep form, then the slot
  // report and its copy to the pinned host table, as one graph.
  rewl_status capture(Group& g, int form) {
    if (g.exec) {
      cudaGraphExecDestroy(g.exec);
      g.exec = nullptr;
    }
    const BatchWalker* list = form == kBatchQuad ? g.d_list + g.n_list : g.d_list;
    const int n = form == kBatchQuad ? g.n_quad : g.n_list;
    const size_t smem = form == kBatchQuad ? g.smem_quad : g.smem;
    cudaGraph_t graph = nullptr;
    SCUDA(cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < g.k && e == cudaSuccess; ++r)
      e = launch_round_batch(g.d_slots, g.hi, list, n, smem, g.max_pairs, g.max_m, g.max_h, form, g.model, g.stream);
    if (e == cudaSuccess) e = launch_slot_report(g.d_slots, g.hi, g.d_rep, g.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.h_rep, g.d_rep, sizeof(SlotReport) * g.hi, cudaMemcpyDeviceToHost, g.stream);
    const cudaError_t e2 = cudaStreamEndCapture(g.stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return sfail(REWL_ECUDA, "capture of a group's rounds: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return sfail(REWL_ECUDA, "instantiate a group's rounds: %s", cudaGetErrorString(e));
    g.exec_form = form;
    g.exec_k = g.k;
    return REWL_OK;
  }

  // One round of group g: sweeps, exchanges, clocks, due flatness checks, report.
  rewl_status launch(Group& g) {
    if (g.dirty) {
      rewl_status st = rebuild(g);
      if (st != REWL_OK) return st;
    }
    if (g.n_list == 0) return REWL_OK;
    // few walkers on the GPU: each walker's chain has a sub-partition to itself, and a producer
    // warp per walker makes its draws (the ring form); many walkers share the SMs and their issue
    // slots, and 4 walkers per CTA with 8 lanes each share the instructions of the sequential step
    const bool few = active_walkers() <= 8 * n_sm;
    int form = kBatchOne;
    if (few && g.smem + ring_extra_smem() <= batch_smem_limit()) form = kBatchRing;
    else if (!few && g.smem_quad <= batch_smem_limit()) form = kBatchQuad;
    if (!g.exec || g.exec_form != form || g.exec_k != g.k) {
      rewl_status st = capture(g, form);
      if (st != REWL_OK) return st;
    }
    g.t_launch = Clock::now();
    SCUDA(cudaGraphLaunch(g.exec, g.stream));
    SCUDA(cudaEventRecord(g.ev, g.stream));
    for (int i = 0; i < (int)g.slot_req.size(); ++i) g.launched[i] = i < g.hi ? g.slot_req[i] : 0;
    g.in_flight = true;
    return REWL_OK;
  }

  void release(Request& r) {
    if (r.group >= 0) {
      Group& g = *groups[r.group];
      g.slots[r.slot].active = 0;
      g.slot_req[r.slot] = 0;
      g.dirty = true;
      r.group = r.slot = -1;
      --n_running;
    }
    if (r.ctx) {
      rewl_destroy(r.ctx);
      r.ctx = nullptr;
      in_use -= r.bytes;
    }
  }

  // Reads the report of a finished replay of g; retires requests whose windows are all done.
  void collect(Group& g) {
    g.in_flight = false;
    rounds += g.exec_k;
    {  // rounds per replay: powers of two, so that one replay lasts about kReplayMs (a shared group:
       // its small requests should not wait long for their last round) or kPrivateReplayMs (a
       // private group: fewer host round trips between the long rounds of its one request)
      const double per_round = ms_between(g.t_launch, Clock::now()) / std::max(1, g.exec_k);
      const double target = g.priv ? kPrivateReplayMs : kReplayMs;
      int k = 1;
      while (k < kMaxRoundsPerReplay && per_round * 2 * k <= target) k *= 2;
      g.k = k;
    }
    for (int s = 0; s < g.hi; ++s) {
      if (!g.slot_req[s] || g.launched[s] != g.slot_req[s]) continue;  // not in that round
      Request& r = reqs[g.slot_req[s]];
      const SlotReport& q = g.h_rep[s];
      attempts += (int64_t)q.attempts - r.attempts;
      r.attempts = (int64_t)q.attempts;
      r.sweeps = (int64_t)q.sweeps;
      r.n_done = q.n_done;
      r.ctx->sweep_clock = q.sweeps;
      r.ctx->xround = q.rounds;
      r.ctx->attempts = q.attempts;
      r.ctx->n_done = q.n_done;
      r.active_walkers = (int64_t)(g.slots[s].P.h - q.n_done) * g.slots[s].P.m;
      if (q.n_done < g.slots[s].P.h) continue;
      r.lng.assign(r.ctx->P.n_bins, 0.0);
      const rewl_status st = rewl_get_lng(r.ctx, r.lng.data(), (int32_t)r.lng.size(), &r.n_bins, &r.e_min, &r.e_step);
      r.t_done = Clock::now();
      if (st != REWL_OK) {
        r.state = REWL_REQ_FAILED;
        r.error = st;
        ++failed;
      } else {
        r.state = REWL_REQ_DONE;
        ++finished;
      }
      release(r);
    }
  }

  // Issues a replay for every idle group with running requests, then waits until
  // at least one replay in flight has finished and collects every finished one.
  // The server's lock is released while it waits on the GPU, so that other
  // threads can submit, poll and fetch results meanwhile (groups live on the
  // heap and stay put; a replay is collected by whichever caller finds it done).
  rewl_status step(std::unique_lock<std::mutex>& lk) {
    std::vector<Group*> flight;
    for (auto& gp : groups) {
      Group& g = *gp;
      if (!g.in_flight && g.running() > 0) {
        rewl_status st = launch(g);
        if (st != REWL_OK) return st;
      }
      if (g.in_flight) flight.push_back(&g);
    }
    if (flight.empty()) return REWL_OK;
    const Clock::time_point t0 = Clock::now();
    std::vector<char> ready(flight.size());
    for (long spin = 0;; ++spin) {
      lk.unlock();
      int got = 0;
      cudaError_t bad = cudaSuccess;
      for (size_t i = 0; i < flight.size(); ++i) {
        const cudaError_t e = cudaEventQuery(flight[i]->ev);
        ready[i] = e == cudaSuccess;
        got += ready[i];
        if (e != cudaSuccess && e != cudaErrorNotReady) bad = e;
      }
      if (!got && bad == cudaSuccess && spin > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
      if (bad != cudaSuccess) return sfail(REWL_ECUDA, "round: %s", cudaGetErrorString(bad));
      if (got) {
        // under the lock again: another caller may have collected a replay seen done above and
        // issued the group's next one, so each group is collected only if its latest event is done
        for (size_t i = 0; i < flight.size(); ++i)
          if (ready[i] && flight[i]->in_flight && cudaEventQuery(flight[i]->ev) == cudaSuccess) collect(*flight[i]);
        return REWL_OK;
      }
      if (params.timeout_ms > 0 && ms_between(t0, Clock::now()) > (double)params.timeout_ms)
        return sfail(REWL_ETIMEOUT, "no round finished within %lld ms", (long long)params.timeout_ms);
    }
  }
};

extern "C" {

rewl_status rewl_server_create(rewl_server_handle* out, int64_t device_bytes, int32_t max_running,
                               const rewl_params* params) {
  if (!out) return sfail(REWL_EINVAL, "NULL argument");
  if (device_bytes <= 0 || max_running < 1 || max_running > 65536)
    return sfail(REWL_EINVAL, "device_bytes must be > 0 and max_running in [1, 65536]");
  if (params && (params->window_starts || params->window_widths))
    return sfail(REWL_EINVAL, "a window table is per problem; served requests use the equal partition");
  rewl_server* s = new rewl_server();
  if (params) s->params = *params;
  else rewl_params_default(&s->params);
  s->budget = device_bytes;
  s->max_running = max_running;
  cudaError_t e = prepare_sweep_batch();
  int dev = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
  s->walker_target = s->params.server_walker_target == 0 ? 24LL * s->n_sm
                     : s->params.server_walker_target < 0 ? 0 : s->params.server_walker_target;
  if (e != cudaSuccess) {
    delete s;
    return sfail(REWL_ECUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  *out = s;
  return REWL_OK;
}

rewl_status rewl_server_submit(rewl_server_handle s, const rewl_request* q, uint64_t* id) {
  if (!s || !q || !id) return sfail(REWL_EINVAL, "NULL argument");
  const int L = q->lattice.Lx;
  const int dim = q->lattice.dim;
  if (q->model.kind < 0 || q->model.kind > 3 || (dim != 2 && dim != 3) ||
      (dim == 3) != (q->model.kind == REWL_EA_PM_J_3D) || q->lattice.Lx != q->lattice.Ly ||
      q->lattice.periodic != 1 || L < 2 || L > (dim == 3 ? 64 : 256) || q->windows < 1 ||
      q->walkers_per_window < 1 || q->walkers_per_window > 4096 || !(q->overlap > 0.0 && q->overlap < 1.0))
    return sfail(REWL_EINVAL, "invalid request");
  if (!(q->flatness > 0.0 && q->flatness <= 1.0) || !(q->lnf_final >= 1e-12))
    return sfail(REWL_EINVAL, "flatness must be in (0, 1] and lnf_final >= 1e-12");
  const bool pmj = q->model.kind == REWL_EA_PM_J || q->model.kind == REWL_EA_PM_J_3D;
  if (!pmj && q->couplings) return sfail(REWL_EINVAL, "couplings are only taken by +-J");
  std::lock_guard<std::mutex> lock(s->mu);
  Request r;
  r.id = s->next_id++;
  r.model = q->model;
  r.lattice = q->lattice;
  if (q->couplings) {
    r.couplings.assign(q->couplings, q->couplings + (dim == 3 ? 3LL * L * L * L : 2LL * L * L));
    r.has_couplings = true;
  }
  r.windows = q->windows;
  r.walkers_per_window = q->walkers_per_window;
  r.overlap = q->overlap;
  r.flatness = q->flatness;
  r.lnf_final = q->lnf_final;
  r.seed = q->seed;
  r.bytes = request_bytes(r);
  if (r.bytes > s->budget) return sfail(REWL_ENOMEM, "request needs %lld bytes, budget %lld", (long long)r.bytes, (long long)s->budget);
  r.t_submit = Clock::now();
  s->queue.push_back(r.id);
  *id = r.id;
  s->reqs.emplace(r.id, std::move(r));
  return REWL_OK;
}

rewl_status rewl_server_run(rewl_server_handle s, int32_t max_rounds, rewl_server_stats* stats) {
  if (!s) return sfail(REWL_EINVAL, "NULL handle");
  std::unique_lock<std::mutex> lock(s->mu);
  for (int32_t k = 0; k < max_rounds; ++k) {
    rewl_status st = s->admit();
    if (st != REWL_OK) return st;
    if (s->n_running == 0) break;
    st = s->step(lock);
    if (st != REWL_OK) return st;
  }
  rewl_status st = s->admit();  // fill slots freed by the last rounds
  if (st != REWL_OK) return st;
  if (stats) {
    stats->running = s->n_running;
    stats->queued = (int32_t)s->queue.size();
    stats->finished = s->finished;
    stats->failed = s->failed;
    stats->rounds = s->rounds;
    stats->attempts = s->attempts;
    stats->device_bytes_in_use = s->in_use;
  }
  return REWL_OK;
}

rewl_status rewl_server_poll(rewl_server_handle s, uint64_t id, rewl_request_info* info) {
  if (!s || !info) return sfail(REWL_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(REWL_ENOTFOUND, "request %llu", (unsigned long long)id);
  const Request& r = it->second;
  const Clock::time_point now = Clock::now();
  info->state = r.state;
  info->error = r.error;
  const bool admitted = r.state != REWL_REQ_QUEUED && r.t_admit.time_since_epoch().count() != 0;
  const bool ended = r.state == REWL_REQ_DONE || r.state == REWL_REQ_FAILED || r.state == REWL_REQ_CANCELLED;
  info->queued_ms = ms_between(r.t_submit, admitted ? r.t_admit : (ended ? r.t_done : now));
  info->run_ms = admitted ? ms_between(r.t_admit, ended ? r.t_done : now) : 0.0;
  info->latency_ms = ms_between(r.t_submit, ended ? r.t_done : now);
  info->sweeps = r.sweeps;
  info->attempts = r.attempts;
  info->device_bytes = r.bytes;
  return REWL_OK;
}

rewl_status rewl_server_result(rewl_server_handle s, uint64_t id, double* lng, int32_t capacity, int32_t* n_bins,
                               int32_t* e_min, int32_t* e_step) {
  if (!s || !lng) return sfail(REWL_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(REWL_ENOTFOUND, "request %llu", (unsigned long long)id);
  const Request& r = it->second;
  if (r.state != REWL_REQ_DONE) return sfail(REWL_EBUSY, "request %llu has no result (state %d)", (unsigned long long)id, r.state);
  if (capacity < r.n_bins) return sfail(REWL_EINVAL, "capacity %d < %d bins", capacity, r.n_bins);
  std::memcpy(lng, r.lng.data(), sizeof(double) * r.n_bins);
  if (n_bins) *n_bins = r.n_bins;
  if (e_min) *e_min = r.e_min;
  if (e_step) *e_step = r.e_step;
  return REWL_OK;
}

rewl_status rewl_server_cancel(rewl_server_handle s, uint64_t id) {
  if (!s) return sfail(REWL_EINVAL, "NULL handle");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(REWL_ENOTFOUND, "request %llu", (unsigned long long)id);
  Request& r = it->second;
  if (r.state == REWL_REQ_QUEUED) {
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), id), s->queue.end());
  } else if (r.state == REWL_REQ_RUNNING) {
    Group& g = *s->groups[r.group];
    if (cudaStreamSynchronize(g.stream) != cudaSuccess) return sfail(REWL_ECUDA, "synchronise");
    if (g.in_flight) s->collect(g);  // the round it was part of; the request may finish in it
    if (r.state != REWL_REQ_RUNNING) return REWL_OK;
    s->release(r);
  } else {
    return REWL_OK;  // already finished
  }
  r.state = REWL_REQ_CANCELLED;
  r.t_done = Clock::now();
  return REWL_OK;
}

void rewl_server_destroy(rewl_server_handle s) { delete s; }

}  // extern "C"
