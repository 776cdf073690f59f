// rewl_server.cu -- the served form of REWL: density-of-states requests of
// different models and lattice sizes arrive at any time, are admitted while
// request slots and the device-memory budget allow, and run together.  Each
// round is one launch per model of the sweep kernel over every walker of every
// running request, one batched exchange launch, one clock launch and one
// batched flatness launch; requests that finish are retired (their joined
// ln g is read back) and their memory goes to the queue.  Every request keeps
// its own seed, schedule and state, so its result is bit-identical to the one
// it gets alone (rewl_create + rewl_step).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
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
  int slot = -1;
  int n_done = 0;
  int64_t sweeps = 0, attempts = 0;
  std::vector<double> lng;
  int32_t n_bins = 0, e_min = 0, e_step = 0;
};

// Device bytes a request may use: its per-walker arrays with the widest
// window its energy range allows, plus per-window tables.
int64_t request_bytes(const Request& r) {
  const int L = r.lattice.Lx, N = L * L;
  const bool potts = r.model.kind == REWL_POTTS;
  const int Wr = potts ? (L + 7) / 8 : (L + 31) / 32, Wr1 = (L + 31) / 32;
  const int64_t lat_words = (int64_t)L * Wr;
  const int64_t B = potts ? 2LL * N + 1 : (int64_t)N + 1;
  int64_t w = B;
  if (r.windows > 1)
    w = std::min<int64_t>(B, (int64_t)std::ceil((double)B / (1.0 + (double)(r.windows - 1) * (1.0 - r.overlap))));
  const int64_t nW = (int64_t)r.windows * r.walkers_per_window;
  return nW * (lat_words * 4 + 4 + w * 12 + 3 * 8 + 3 * 4 + 8) + (int64_t)r.windows * 48 + lat_words * 4 +
         2LL * L * Wr1 * 4 + 4096;
}

}  // namespace

struct rewl_server {
  std::mutex mu;
  rewl_params params{};
  int64_t budget = 0, in_use = 0;
  int max_running = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint64_t next_id = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<uint64_t> slot_req;  // request id per slot, 0 = free
  std::vector<BatchSlot> h_slots;
  BatchSlot* d_slots = nullptr;
  BatchWalker* d_lists[3] = {nullptr, nullptr, nullptr};
  int list_cap[3] = {0, 0, 0};
  int n_list[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  int max_pairs = 0, max_m = 1, max_h = 1;
  bool lists_dirty = true;
  int32_t* d_done = nullptr;
  int32_t* h_done = nullptr;  // pinned
  int64_t rounds = 0, attempts = 0;
  int finished = 0, failed = 0;

  ~rewl_server() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto& kv : reqs)
      if (kv.second.ctx) rewl_destroy(kv.second.ctx);
    cudaFree(d_slots);
    for (int k = 0; k < 3; ++k) cudaFree(d_lists[k]);
    cudaFree(d_done);
    if (h_done) cudaFreeHost(h_done);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  int running() const {
    int n = 0;
    for (uint64_t id : slot_req) n += id != 0;
    return n;
  }

  rewl_status upload_slot(int s) {
    SCUDA(cudaMemcpyAsync(d_slots + s, &h_slots[s], sizeof(BatchSlot), cudaMemcpyHostToDevice, stream));
    return REWL_OK;
  }

  // Admission: first-come first-served while a slot and the memory budget allow.
  rewl_status admit() {
    while (!queue.empty()) {
      const uint64_t id = queue.front();
      Request& r = reqs[id];
      int s = -1;
      for (int i = 0; i < max_running; ++i)
        if (!slot_req[i]) {
          s = i;
          break;
        }
      if (s < 0 || in_use + r.bytes > budget) break;  // head of queue waits for capacity
      queue.pop_front();
      rewl_params p = params;
      p.stream = (void*)stream;
      p.lanes_per_walker = 32;
      p.walkers_per_block = 1;
      p.mode = REWL_MODE_PLAIN;
      p.profile = 0;
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
      r.ctx = h;
      r.slot = s;
      r.state = REWL_REQ_RUNNING;
      r.t_admit = Clock::now();
      in_use += r.bytes;
      slot_req[s] = id;
      BatchSlot& b = h_slots[s];
      b.P = h->P;
      b.S = h->S;
      b.spe = (uint32_t)h->params.sweeps_per_exchange;
      b.spf = (uint32_t)h->params.sweeps_per_flat_check;
      b.n_att = b.spe * (uint32_t)h->P.N;
      b.active = 1;
      rewl_status us = upload_slot(s);
      if (us != REWL_OK) return us;
      lists_dirty = true;
    }
    return REWL_OK;
  }

  rewl_status rebuild_lists() {
    std::vector<BatchWalker> L[3];
    max_pairs = 0;
    max_m = 1;
    max_h = 1;
    for (int k = 0; k < 3; ++k) smem[k] = 0;
    for (int s = 0; s < max_running; ++s) {
      if (!slot_req[s]) continue;
      const Problem& P = h_slots[s].P;
      for (int W = 0; W < P.n_walkers; ++W) L[P.model].push_back(BatchWalker{s, W});
      smem[P.model] = std::max(smem[P.model], sweep_smem_bytes(P, 1, 32, kSweepChain));
      max_pairs = std::max(max_pairs, P.h / 2);
      max_m = std::max(max_m, P.m);
      max_h = std::max(max_h, P.h);
    }
    for (int k = 0; k < 3; ++k) {
      n_list[k] = (int)L[k].size();
      if (n_list[k] > list_cap[k]) {
        cudaFree(d_lists[k]);
        d_lists[k] = nullptr;
        const int cap = std::max(n_list[k], 2 * list_cap[k]);
        if (cudaMalloc(&d_lists[k], sizeof(BatchWalker) * cap) != cudaSuccess) {
          list_cap[k] = 0;
          return sfail(REWL_ENOMEM, "walker list of %d entries", cap);
        }
        list_cap[k] = cap;
      }
      if (n_list[k])
        SCUDA(cudaMemcpyAsync(d_lists[k], L[k].data(), sizeof(BatchWalker) * n_list[k], cudaMemcpyHostToDevice, stream));
    }
    lists_dirty = false;
    return REWL_OK;
  }

  void release(Request& r) {
    if (r.slot >= 0) {
      h_slots[r.slot].active = 0;
      upload_slot(r.slot);
      slot_req[r.slot] = 0;
      r.slot = -1;
      lists_dirty = true;
    }
    if (r.ctx) {
      rewl_destroy(r.ctx);
      r.ctx = nullptr;
      in_use -= r.bytes;
    }
  }

  rewl_status round() {
    if (lists_dirty) {
      rewl_status st = rebuild_lists();
      if (st != REWL_OK) return st;
    }
    // walkers of windows still running: what this round's sweeps count
    for (int s = 0; s < max_running; ++s) {
      if (!slot_req[s]) continue;
      Request& r = reqs[slot_req[s]];
      const Problem& P = h_slots[s].P;
      const int64_t n = (int64_t)(P.h - r.n_done) * P.m * h_slots[s].spe * P.N;
      r.attempts += n;
      attempts += n;
      r.sweeps += h_slots[s].spe;
      r.ctx->attempts += (uint64_t)n;
      r.ctx->sweep_clock += h_slots[s].spe;
      r.ctx->xround += 1;
    }
    SCUDA(launch_round_batch(d_slots, max_running, d_lists, n_list, smem, max_pairs, max_m, max_h, stream));
    SCUDA(launch_gather_done(d_slots, max_running, d_done, stream));
    SCUDA(cudaMemcpyAsync(h_done, d_done, sizeof(int32_t) * max_running, cudaMemcpyDeviceToHost, stream));
    SCUDA(cudaStreamSynchronize(stream));
    ++rounds;
    for (int s = 0; s < max_running; ++s) {
      if (!slot_req[s]) continue;
      Request& r = reqs[slot_req[s]];
      r.n_done = h_done[s];
      r.ctx->n_done = h_done[s];
      if (h_done[s] < h_slots[s].P.h) continue;
      // finished: read the joined ln g back, then free the slot and memory
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
    return REWL_OK;
  }
};

static double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

extern "C" {

rewl_status rewl_server_create(rewl_server_handle* out, int64_t device_bytes, int32_t max_running,
                               const rewl_params* params) {
  if (!out) return sfail(REWL_EINVAL, "NULL argument");
  if (device_bytes <= 0 || max_running < 1 || max_running > 65536)
    return sfail(REWL_EINVAL, "device_bytes must be > 0 and max_running in [1, 65536]");
  rewl_server* s = new rewl_server();
  if (params) s->params = *params;
  else rewl_params_default(&s->params);
  s->budget = device_bytes;
  s->max_running = max_running;
  s->slot_req.assign(max_running, 0);
  s->h_slots.assign(max_running, BatchSlot{});
  auto bail = [&](rewl_status st) {
    delete s;
    return st;
  };
  if (s->params.stream) {
    s->stream = (cudaStream_t)s->params.stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(sfail(REWL_ECUDA, "cudaStreamCreate failed"));
    s->own_stream = true;
  }
  if (cudaMalloc(&s->d_slots, sizeof(BatchSlot) * max_running) != cudaSuccess ||
      cudaMalloc(&s->d_done, sizeof(int32_t) * max_running) != cudaSuccess ||
      cudaMallocHost(&s->h_done, sizeof(int32_t) * max_running) != cudaSuccess)
    return bail(sfail(REWL_ENOMEM, "server tables"));
  cudaError_t e = cudaMemsetAsync(s->d_slots, 0, sizeof(BatchSlot) * max_running, s->stream);
  if (e == cudaSuccess) e = prepare_sweep_batch();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return bail(sfail(REWL_ECUDA, "server set-up: %s", cudaGetErrorString(e)));
  *out = s;
  return REWL_OK;
}

rewl_status rewl_server_submit(rewl_server_handle s, const rewl_request* q, uint64_t* id) {
  if (!s || !q || !id) return sfail(REWL_EINVAL, "NULL argument");
  const int L = q->lattice.Lx;
  if (q->model.kind < 0 || q->model.kind > 2 || q->lattice.dim != 2 || q->lattice.Lx != q->lattice.Ly ||
      q->lattice.periodic != 1 || L < 2 || L > 128 || q->windows < 1 || q->walkers_per_window < 1 ||
      q->walkers_per_window > 4096 || !(q->overlap > 0.0 && q->overlap < 1.0))
    return sfail(REWL_EINVAL, "invalid request");
  if (q->model.kind != REWL_EA_PM_J && q->couplings) return sfail(REWL_EINVAL, "couplings are only taken by +-J");
  std::lock_guard<std::mutex> lock(s->mu);
  Request r;
  r.id = s->next_id++;
  r.model = q->model;
  r.lattice = q->lattice;
  if (q->couplings) {
    r.couplings.assign(q->couplings, q->couplings + 2 * L * L);
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
  std::lock_guard<std::mutex> lock(s->mu);
  for (int32_t k = 0; k < max_rounds; ++k) {
    rewl_status st = s->admit();
    if (st != REWL_OK) return st;
    if (s->running() == 0) break;
    st = s->round();
    if (st != REWL_OK) return st;
  }
  rewl_status st = s->admit();  // fill slots freed by the last round
  if (st != REWL_OK) return st;
  if (stats) {
    stats->running = s->running();
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
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return sfail(REWL_ECUDA, "synchronise");
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
