// rewl_host.cu -- host runtime of the REWL library and its C ABI
// (include/rewl.h): validation, energy bins and windows, device memory,
// set-up, the phase schedule (plain launches or a captured CUDA graph per
// flatness period), joining of the window fragments, state access.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rewl.h"
#include "rewl_ctx.h"
#include "rewl_device.cuh"
#include "rewl_kernels.h"
#include "rewl_layout.h"

using namespace rewl;

namespace {

thread_local std::string g_last_error = "";

rewl_status fail(rewl_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (expr);                                                                            \
    if (e_ != cudaSuccess) return fail(REWL_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

}  // namespace

void* rewl_ctx::dalloc(size_t bytes, rewl_status* st) {
  void* p = nullptr;
  bytes = std::max<size_t>(bytes, 16);
  if (params.alloc) {
    p = params.alloc(bytes, (void*)stream, params.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (!p) {
    *st = fail(REWL_ENOMEM, "device allocation of %zu bytes failed", bytes);
    return nullptr;
  }
  allocations.push_back(p);
  return p;
}

rewl_ctx::~rewl_ctx() {
  if (stream) cudaStreamSynchronize(stream);
  if (graph) cudaGraphExecDestroy(graph);
  for (void* p : allocations) {
    if (params.free) params.free(p, (void*)stream, params.alloc_user);
    else cudaFree(p);
  }
  if (pre_stream) cudaStreamSynchronize(pre_stream);
  if (h_n_done) cudaFreeHost(h_n_done);
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    if (ev_pre[k]) cudaEventDestroy(ev_pre[k]);
    if (ev_used[k]) cudaEventDestroy(ev_used[k]);
  }
  if (pre_stream) cudaStreamDestroy(pre_stream);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

// ---------------------------------------------------------------------------
// Energy windows: w = ceil(B / (1 + (h-1)(1-o))) bins, window k starting at
// k(B-w)/(h-1) rounded half up (paper, Fig. 1a: equal-size windows, overlap o).
// ---------------------------------------------------------------------------
// The equal partition covers the core bins [core_lo, core_lo + Bc) (all B bins
// but for +-J, where the core is the descent's range); the first and the last
// window then reach down to bin 0 and up to bin B-1.
static rewl_status make_windows(int B, int h, double o, int core_lo, int Bc, int* w_out, std::vector<int32_t>& start,
                                std::vector<int32_t>& width) {
  start.assign(h, 0);
  if (h == 1) {
    *w_out = B;
    width.assign(1, B);
    return REWL_OK;
  }
  int w = (int)std::ceil((double)Bc / (1.0 + (double)(h - 1) * (1.0 - o)));
  if (w > Bc) w = Bc;
  if (w < 3) return fail(REWL_EINVAL, "windows of %d bins are too narrow (B=%d, h=%d)", w, Bc, h);
  for (int k = 0; k < h; ++k) start[k] = core_lo + (int32_t)((2LL * k * (Bc - w) + (h - 1)) / (2LL * (h - 1)));
  for (int k = 0; k + 1 < h; ++k)
    if (start[k + 1] > start[k] + w - 1) return fail(REWL_EINVAL, "windows %d and %d do not overlap", k, k + 1);
  width.assign(h, w);
  width[0] += start[0];
  start[0] = 0;
  width[h - 1] = B - start[h - 1];
  *w_out = *std::max_element(width.begin(), width.end());
  return REWL_OK;
}

// An explicit partition (Fig. 1b: run-time balanced windows of unequal width):
// from bin 0 to bin B-1, widths >= 3, starts and ends strictly increasing,
// neighbours sharing at least one bin.
static rewl_status check_windows(int B, int h, const int32_t* st, const int32_t* wd) {
  if (st[0] != 0 || (int64_t)st[h - 1] + wd[h - 1] != B)
    return fail(REWL_EINVAL, "the windows must cover bins 0 .. %d", B - 1);
  for (int k = 0; k < h; ++k) {
    if (wd[k] < 3 || st[k] < 0 || (int64_t)st[k] + wd[k] > B) return fail(REWL_EINVAL, "window %d: start %d width %d", k, st[k], wd[k]);
    if (k > 0 && (st[k] <= st[k - 1] || st[k] + wd[k] <= st[k - 1] + wd[k - 1]))
      return fail(REWL_EINVAL, "windows %d and %d are not ordered", k - 1, k);
    if (k > 0 && st[k] > st[k - 1] + wd[k - 1] - 1) return fail(REWL_EINVAL, "windows %d and %d do not overlap", k - 1, k);
  }
  return REWL_OK;
}

static bool is_pow2_double(double v) {
  if (!(v > 0.0) || !std::isfinite(v)) return false;
  int e;
  const double m = std::frexp(v, &e);
  return m == 0.5;
}

// Kernel configuration: G lanes per walker and walkers per CTA.  Few walkers
// run latency-bound (one sequential chain each), so they get whole warps and
// are spread over all SMs; many walkers share warps.
static void choose_config(rewl_ctx* c, int n_sm) {
  const Problem& P = c->P;
  int G = c->params.lanes_per_walker;
  if (G == 0) {
    const int nw = P.n_walkers;
    if (nw <= 8 * n_sm) G = 32;
    else if (nw <= 32 * n_sm) G = 8;
    else G = 4;
  }
  int wpb = c->params.walkers_per_block;
  if (wpb == 0) {
    wpb = std::max(1, 256 / G);
    const size_t budget = 200 * 1024;
    while (wpb > 1 && sweep_smem_bytes(P, wpb, G, c->params.sweep_variant) > budget) --wpb;
    const int spread = (P.n_walkers + n_sm - 1) / n_sm;  // at least one CTA per SM when possible
    wpb = std::max(1, std::min(wpb, spread));
  }
  wpb = std::max(1, std::min(wpb, 256 / G));
  if (c->params.sweep_variant == kSweepRing) {  // one walker per CTA on a whole warp, plus its producer warp
    G = 32;
    wpb = 1;
  }
  c->G = G;
  c->wpb = wpb;
}

// Counted copies (the e2e accounting of rewl_info.h2d_bytes / d2h_bytes).
static cudaError_t h2d(rewl_ctx* c, void* dst, const void* src, size_t n) {
  c->h2d_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->stream);
}
static cudaError_t d2h(rewl_ctx* c, void* dst, const void* src, size_t n) {
  c->d2h_bytes += n;
  return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->stream);
}

// Folds the timed sweep launches since the last synchronisation into the totals.
static rewl_status collect_sweep_times(rewl_ctx* c) {
  for (int i = 0; i < c->ev_pending; ++i) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
    c->sweep_ms += ms;
    c->sweep_launches += 1;
  }
  c->ev_pending = 0;
  return REWL_OK;
}

static rewl_status upload_active(rewl_ctx* c) {
  std::vector<int32_t> done(c->P.h), act;
  CUDA_TRY(d2h(c, done.data(), c->S.done, sizeof(int32_t) * c->P.h));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  int nd = 0;
  for (int a = 0; a < c->P.h; ++a) {
    nd += done[a] != 0;
    if (!done[a])
      for (int k = 0; k < c->P.m; ++k) act.push_back(a * c->P.m + k);
  }
  c->n_done = nd;
  c->n_active = (int)act.size();
  if (!act.empty())
    CUDA_TRY(h2d(c, c->S.active, act.data(), sizeof(int32_t) * act.size()));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return REWL_OK;
}

static rewl_status check_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(REWL_ENODEV, "no CUDA device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(REWL_ENODEV, "no CUDA device");
  if (prop.major != 10 || prop.minor != 3)
    return fail(REWL_ENODEV, "device %s is sm_%d%d; this library is built for sm_103a", prop.name, prop.major,
                prop.minor);
  return REWL_OK;
}

extern "C" {

void rewl_params_default(rewl_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->sweeps_per_exchange = 100;
  p->sweeps_per_flat_check = 1000;
  p->lnf0 = 1.0;
  p->entry_max_sweeps = 1000;
  p->discovery_sweeps = 200;
  p->mode = REWL_MODE_PLAIN;
  p->sweep_variant = REWL_SWEEP_AUTO;
}

const char* rewl_status_str(rewl_status s) {
  switch (s) {
    case REWL_OK: return "ok";
    case REWL_EINVAL: return "invalid argument";
    case REWL_ENOMEM: return "out of memory";
    case REWL_ECUDA: return "CUDA error";
    case REWL_ETIMEOUT: return "timeout";
    case REWL_EENTRY: return "a walker could not enter its energy window";
    case REWL_EOVERFLOW: return "histogram overflow";
    case REWL_EBUSY: return "busy";
    case REWL_ENOTFOUND: return "not found";
    case REWL_ENODEV: return "no suitable CUDA device";
  }
  return "unknown status";
}

const char* rewl_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// Lets the other translation units of the library report through rewl_last_error.
void rewl_set_last_error(const char* msg) { g_last_error = msg; }

extern "C" {

rewl_status rewl_create(rewl_handle* out, const rewl_model* model, const rewl_lattice* lattice,
                        const int8_t* couplings, int32_t windows, double overlap, int32_t walkers_per_window,
                        double flatness, double lnf_final, uint64_t seed, const rewl_params* params) {
  if (!out || !model || !lattice) return fail(REWL_EINVAL, "NULL argument");
  rewl_params prm;
  if (params) prm = *params;
  else rewl_params_default(&prm);
  const int kind = model->kind;
  if (kind < 0 || kind > 3) return fail(REWL_EINVAL, "unknown model kind %d", kind);
  if (kind == REWL_POTTS && (model->q < 2 || model->q > 16)) return fail(REWL_EINVAL, "Potts q=%d not in [2,16]", model->q);
  const int dim = lattice->dim;
  if ((dim != 2 && dim != 3) || lattice->Lx != lattice->Ly || lattice->periodic != 1 ||
      (dim == 3) != (kind == REWL_EA_PM_J_3D))
    return fail(REWL_EINVAL, "periodic square lattices, or the periodic cube for the 3D +-J model");
  const int L = lattice->Lx;
  if (L < 2 || L > (dim == 3 ? 64 : 256)) return fail(REWL_EINVAL, "L=%d not in [2,%d]", L, dim == 3 ? 64 : 256);
  const bool pmj = kind == REWL_EA_PM_J || kind == REWL_EA_PM_J_3D;
  if (pmj && (L % 2)) return fail(REWL_EINVAL, "+-J needs an even L");
  if (!pmj && couplings) return fail(REWL_EINVAL, "couplings are only taken by the +-J models");
  const int64_t N64 = dim == 3 ? (int64_t)L * L * L : (int64_t)L * L;
  if (windows < 1 || walkers_per_window < 1 || walkers_per_window > 4096 ||
      (int64_t)windows * walkers_per_window > (1 << 20))
    return fail(REWL_EINVAL, "windows=%d walkers_per_window=%d", windows, walkers_per_window);
  if (!(overlap > 0.0 && overlap < 1.0)) return fail(REWL_EINVAL, "overlap %g not in (0,1)", overlap);
  if (!(flatness > 0.0 && flatness <= 1.0)) return fail(REWL_EINVAL, "flatness %g not in (0,1]", flatness);
  if (!(lnf_final > 0.0) || lnf_final < 1e-12) return fail(REWL_EINVAL, "lnf_final %g must be in [1e-12, ...)", lnf_final);
  if (!is_pow2_double(prm.lnf0) || !(prm.lnf0 >= lnf_final) || prm.lnf0 > 64.0)
    return fail(REWL_EINVAL, "lnf0 %g must be a power of two in [lnf_final, 64]", prm.lnf0);
  if (prm.sweeps_per_exchange < 1 || prm.sweeps_per_flat_check < prm.sweeps_per_exchange ||
      prm.sweeps_per_flat_check % prm.sweeps_per_exchange != 0)
    return fail(REWL_EINVAL, "sweeps_per_flat_check must be a positive multiple of sweeps_per_exchange");
  if ((int64_t)prm.sweeps_per_exchange * N64 > 0x7fffffffLL) return fail(REWL_EINVAL, "sweeps_per_exchange too large");
  if (prm.entry_max_sweeps < 1 || prm.discovery_sweeps < 0) return fail(REWL_EINVAL, "entry/discovery sweeps");
  const int G = prm.lanes_per_walker;
  if (G != 0 && G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32)
    return fail(REWL_EINVAL, "lanes_per_walker %d", G);
  if (prm.walkers_per_block < 0 || (G && prm.walkers_per_block * G > 256))
    return fail(REWL_EINVAL, "walkers_per_block %d", prm.walkers_per_block);
  if (prm.mode != REWL_MODE_PLAIN && prm.mode != REWL_MODE_GRAPH) return fail(REWL_EINVAL, "mode %d", prm.mode);
  if (prm.sweep_variant < REWL_SWEEP_AUTO || prm.sweep_variant > kSweepRing)
    return fail(REWL_EINVAL, "sweep_variant %d", prm.sweep_variant);
  if (prm.sweep_variant == kSweepRing && ((prm.lanes_per_walker != 0 && prm.lanes_per_walker != 32) ||
                                          prm.walkers_per_block > 1))
    return fail(REWL_EINVAL, "the ring variant runs 32 lanes and one walker per CTA");
  if (prm.wl_rule != REWL_RULE_FLAT && prm.wl_rule != REWL_RULE_ONE_OVER_T) return fail(REWL_EINVAL, "wl_rule %d", prm.wl_rule);
  if ((prm.window_starts == nullptr) != (prm.window_widths == nullptr))
    return fail(REWL_EINVAL, "window_starts and window_widths go together");
  if (prm.prefetch_draws != 0 && prm.prefetch_draws != 1) return fail(REWL_EINVAL, "prefetch_draws %d", prm.prefetch_draws);
  if (prm.wait_cycles < 0 || prm.wait_cycles > (1ll << 40)) return fail(REWL_EINVAL, "wait_cycles %lld", (long long)prm.wait_cycles);
  if (couplings)
    for (int64_t i = 0; i < dim * N64; ++i)
      if (couplings[i] != 1 && couplings[i] != -1) return fail(REWL_EINVAL, "coupling %lld is %d", (long long)i, couplings[i]);
  rewl_status st = check_device();
  if (st != REWL_OK) return st;

  rewl_ctx* c = new rewl_ctx();
  c->params = prm;
  c->overlap = overlap;
  Problem& P = c->P;
  P.model = kind;
  P.q = kind == REWL_POTTS ? model->q : 2;
  P.L = L;
  P.N = (int)N64;
  P.rows = dim == 3 ? L * L : L;
  P.Wr = kind == REWL_POTTS ? (L + 7) / 8 : (L + 31) / 32;
  P.Wr1 = (L + 31) / 32;
  P.lat_words = P.rows * P.Wr;
  P.j_words = dim * P.rows * P.Wr1;
  P.magic_L2 = (uint32_t)(((1ull << 32) + (uint64_t)L * L - 1) / ((uint64_t)L * L));
  P.h = windows;
  P.m = walkers_per_window;
  P.n_walkers = windows * walkers_per_window;
  P.magic_L = (uint32_t)(((1ull << 32) + (uint64_t)L - 1) / (uint64_t)L);
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  P.flatness = flatness;
  P.wl_rule = prm.wl_rule;
  P.lnf_final = lnf_final;

  auto bail = [&](rewl_status s) {
    delete c;
    return s;
  };
  if (prm.stream) {
    c->stream = (cudaStream_t)prm.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(fail(REWL_ECUDA, "cudaStreamCreate failed"));
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->h_n_done, 2 * sizeof(int32_t)) != cudaSuccess) return bail(fail(REWL_ENOMEM, "pinned alloc"));

  // couplings: given, or drawn with p = 1/2 (bond b = dim i + d of site i,
  // bit b of the coupling stream), packed as bit planes (bit 1 = J = -1)
  const int nJ = P.j_words;
  std::vector<uint32_t> Jbits(nJ, 0u);
  if (pmj) {
    for (int i = 0; i < P.N; ++i) {
      const int x = i % L, row = i / L;
      for (int d = 0; d < dim; ++d) {
        bool neg;
        if (couplings) {
          neg = couplings[(int64_t)dim * i + d] < 0;
        } else {
          const int b = dim * i + d;
          const U4 r = philox10((uint32_t)(b / 128), 0u, 0xFFFFFFFFu, kTagCoupling, P.seed_lo, P.seed_hi);
          const int wi = (b % 128) / 32;
          const uint32_t wd = wi == 0 ? r.x : wi == 1 ? r.y : wi == 2 ? r.z : r.w;
          neg = (wd >> (b % 32)) & 1u;
        }
        if (neg) Jbits[(d * P.rows + row) * P.Wr1 + (x >> 5)] |= 1u << (x & 31);
      }
    }
  }

  // device memory that does not depend on the window width
  const int nW = P.n_walkers;
  DevState& S = c->S;
  S.lat = (uint32_t*)c->dalloc(sizeof(uint32_t) * (size_t)nW * P.lat_words, &st);
  S.J = (uint32_t*)c->dalloc(sizeof(uint32_t) * nJ, &st);
  S.E = (int32_t*)c->dalloc(sizeof(int32_t) * nW, &st);
  S.win_start = (int32_t*)c->dalloc(sizeof(int32_t) * P.h, &st);
  S.win_width = (int32_t*)c->dalloc(sizeof(int32_t) * P.h, &st);
  S.first_iter = (int64_t*)c->dalloc(sizeof(int64_t) * P.h, &st);
  S.rep_id = (int32_t*)c->dalloc(sizeof(int32_t) * P.n_walkers, &st);
  S.rep_state = (int32_t*)c->dalloc(sizeof(int32_t) * P.n_walkers, &st);
  S.rep_trips = (int64_t*)c->dalloc(sizeof(int64_t) * P.n_walkers, &st);
  S.lnf = (double*)c->dalloc(sizeof(double) * P.h, &st);
  S.iter = (int32_t*)c->dalloc(sizeof(int32_t) * P.h, &st);
  S.done = (int32_t*)c->dalloc(sizeof(int32_t) * P.h, &st);
  S.stage = (int32_t*)c->dalloc(sizeof(int32_t) * P.h, &st);
  S.n_done = (int32_t*)c->dalloc(2 * sizeof(int32_t), &st);  // [0] windows done, [1] the error word
  S.wl_accept = (uint64_t*)c->dalloc(sizeof(uint64_t) * nW, &st);
  S.near_ties = (uint64_t*)c->dalloc(sizeof(uint64_t) * nW, &st);
  S.exact_tests = (uint64_t*)c->dalloc(sizeof(uint64_t) * nW, &st);
  S.x_tried = (uint64_t*)c->dalloc(sizeof(uint64_t) * P.h, &st);
  S.x_accepted = (uint64_t*)c->dalloc(sizeof(uint64_t) * P.h, &st);
  S.active = (int32_t*)c->dalloc(sizeof(int32_t) * nW, &st);
  S.status = (int32_t*)c->dalloc(sizeof(int32_t) * nW, &st);
  S.entry_t = (uint64_t*)c->dalloc(sizeof(uint64_t) * nW, &st);
  S.seed_config = (uint32_t*)c->dalloc(sizeof(uint32_t) * P.lat_words, &st);
  S.clock = (uint64_t*)c->dalloc(sizeof(uint64_t) * 3, &st);
  if (st != REWL_OK) return bail(st);
  cudaStream_t s = c->stream;
#define BAIL_CUDA(expr)                                                                                   \
  do {                                                                                                    \
    cudaError_t e_ = (expr);                                                                              \
    if (e_ != cudaSuccess) return bail(fail(REWL_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)));        \
  } while (0)
  BAIL_CUDA(h2d(c, S.J, Jbits.data(), sizeof(uint32_t) * nJ));
  {  // every walker starts with its own replica; those of the lowest window have been there
    std::vector<int32_t> id(nW), stt(nW);
    for (int W = 0; W < nW; ++W) {
      id[W] = W;
      stt[W] = W < P.m ? 1 : 0;
    }
    BAIL_CUDA(h2d(c, S.rep_id, id.data(), sizeof(int32_t) * nW));
    BAIL_CUDA(h2d(c, S.rep_state, stt.data(), sizeof(int32_t) * nW));
    BAIL_CUDA(cudaMemsetAsync(S.rep_trips, 0, sizeof(int64_t) * nW, s));
  }
  S.error = S.n_done + 1;
  BAIL_CUDA(cudaMemsetAsync(S.n_done, 0, 2 * sizeof(int32_t), s));
  BAIL_CUDA(cudaMemsetAsync(S.iter, 0, sizeof(int32_t) * P.h, s));
  BAIL_CUDA(cudaMemsetAsync(S.done, 0, sizeof(int32_t) * P.h, s));
  BAIL_CUDA(cudaMemsetAsync(S.stage, 0, sizeof(int32_t) * P.h, s));
  BAIL_CUDA(cudaMemsetAsync(S.wl_accept, 0, sizeof(uint64_t) * nW, s));
  BAIL_CUDA(cudaMemsetAsync(S.near_ties, 0, sizeof(uint64_t) * nW, s));
  BAIL_CUDA(cudaMemsetAsync(S.exact_tests, 0, sizeof(uint64_t) * nW, s));
  BAIL_CUDA(cudaMemsetAsync(S.x_tried, 0, sizeof(uint64_t) * P.h, s));
  BAIL_CUDA(cudaMemsetAsync(S.x_accepted, 0, sizeof(uint64_t) * P.h, s));
  BAIL_CUDA(cudaMemsetAsync(S.seed_config, 0, sizeof(uint32_t) * P.lat_words, s));
  BAIL_CUDA(cudaMemsetAsync(S.clock, 0, sizeof(uint64_t) * 3, s));
  BAIL_CUDA(launch_init(P, S, s));

  // energy range
  int core_lo = 0, core_bins = 0;
  if (kind == REWL_ISING) {
    P.e_min = -2 * P.N;
    c->e_max = 2 * P.N;
    P.e_step = 4;
  } else if (kind == REWL_POTTS) {
    P.e_min = -2 * P.N;
    c->e_max = 0;
    P.e_step = 1;
  } else {
    P.e_step = 4;
    BAIL_CUDA(launch_descent(P, S, (uint64_t)prm.discovery_sweeps * P.N, s));
    std::vector<int32_t> E(nW);
    BAIL_CUDA(d2h(c, E.data(), S.E, sizeof(int32_t) * nW));
    BAIL_CUDA(cudaStreamSynchronize(s));
    int best = E[0], bw = 0;
    for (int W = 1; W < nW; ++W)
      if (E[W] < best) best = E[W], bw = W;
    if (best >= 0) return bail(fail(REWL_EENTRY, "descent found no negative energy"));
    // windows over the descent's range [best, -best]; the grid, and the lowest and highest
    // window, reach on to >= -dim N in steps of 4 so that lower energies can still be found
    core_lo = (best + dim * P.N) / 4;
    core_bins = (-2 * best) / 4 + 1;
    P.e_min = best - 4 * core_lo;
    c->e_max = -P.e_min;
    BAIL_CUDA(cudaMemcpyAsync(S.seed_config, S.lat + (size_t)bw * P.lat_words, sizeof(uint32_t) * P.lat_words,
                              cudaMemcpyDeviceToDevice, s));
  }
  P.n_bins = (c->e_max - P.e_min) / P.e_step + 1;
  if (core_bins == 0) core_bins = P.n_bins;
  if (prm.window_starts) {
    st = check_windows(P.n_bins, P.h, prm.window_starts, prm.window_widths);
    if (st != REWL_OK) return bail(st);
    c->win_start.assign(prm.window_starts, prm.window_starts + P.h);
    c->win_width.assign(prm.window_widths, prm.window_widths + P.h);
    P.w = *std::max_element(c->win_width.begin(), c->win_width.end());
  } else {
    st = make_windows(P.n_bins, P.h, overlap, core_lo, core_bins, &P.w, c->win_start, c->win_width);
    if (st != REWL_OK) return bail(st);
  }
  S.lng = (double*)c->dalloc(sizeof(double) * (size_t)nW * P.w, &st);
  S.H = (uint32_t*)c->dalloc(sizeof(uint32_t) * (size_t)nW * P.w, &st);
  if (st != REWL_OK) return bail(st);
  std::vector<double> lnf(P.h, prm.lnf0);
  BAIL_CUDA(h2d(c, S.win_start, c->win_start.data(), sizeof(int32_t) * P.h));
  BAIL_CUDA(h2d(c, S.win_width, c->win_width.data(), sizeof(int32_t) * P.h));
  {
    const std::vector<int64_t> none(P.h, -1);
    BAIL_CUDA(h2d(c, S.first_iter, none.data(), sizeof(int64_t) * P.h));
  }
  BAIL_CUDA(h2d(c, S.lnf, lnf.data(), sizeof(double) * P.h));
  BAIL_CUDA(cudaMemsetAsync(S.lng, 0, sizeof(double) * (size_t)nW * P.w, s));
  BAIL_CUDA(cudaMemsetAsync(S.H, 0, sizeof(uint32_t) * (size_t)nW * P.w, s));
  BAIL_CUDA(launch_entry(P, S, (uint64_t)prm.entry_max_sweeps * P.N, s));
  std::vector<int32_t> status(nW);
  BAIL_CUDA(d2h(c, status.data(), S.status, sizeof(int32_t) * nW));
  BAIL_CUDA(cudaStreamSynchronize(s));
  for (int W = 0; W < nW; ++W)
    if (status[W]) return bail(fail(REWL_EENTRY, "walker %d could not enter window %d", W, W / P.m));
  int dev = 0, n_sm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (c->params.sweep_variant == REWL_SWEEP_AUTO) {
    // latency-bound solves (few walkers: each gets a whole warp on its own SM) run the chain with a
    // producer warp; many walkers share SMs, where the producer's issue slots would come out of
    // other walkers' chains, and run the plain chain
    const bool own_sm = P.n_walkers <= 8 * n_sm && (prm.lanes_per_walker == 0 || prm.lanes_per_walker == 32) &&
                        prm.walkers_per_block <= 1;
    c->params.sweep_variant = own_sm ? kSweepRing : kSweepChain;
  }
  choose_config(c, n_sm);
  c->n_sm = n_sm;
  BAIL_CUDA(prepare_sweep(c->G, P.model));
  // Draws prepared ahead on the idle SMs: plain mode, chain kernel, G >= 8, both buffers within 1 GiB.
  {
    const uint64_t n_att = (uint64_t)prm.sweeps_per_exchange * P.N;
    const uint64_t stride = (n_att + 31) / 32 * 32;
    const uint64_t bytes = (uint64_t)P.n_walkers * stride * sizeof(PreTrial);
    if (prm.prefetch_draws == 1 && prm.mode == REWL_MODE_PLAIN && c->params.sweep_variant == kSweepChain && c->G >= 8 &&
        2 * bytes <= (1ull << 30)) {
      c->pre_stride = (uint32_t)stride;
      c->pre_buf[0] = (PreTrial*)c->dalloc(bytes, &st);
      c->pre_buf[1] = (PreTrial*)c->dalloc(bytes, &st);
      if (st != REWL_OK) return bail(st);
      BAIL_CUDA(cudaStreamCreateWithFlags(&c->pre_stream, cudaStreamNonBlocking));
      for (int k = 0; k < 2; ++k) {
        BAIL_CUDA(cudaEventCreateWithFlags(&c->ev_pre[k], cudaEventDisableTiming));
        BAIL_CUDA(cudaEventCreateWithFlags(&c->ev_used[k], cudaEventDisableTiming));
      }
      c->pre_on = true;
    }
  }
  if (sweep_smem_bytes(P, c->wpb, c->G, c->params.sweep_variant) > 227 * 1024)
    return bail(fail(REWL_EINVAL, "a walker needs %zu bytes of shared memory (window of %d bins)",
                     sweep_smem_bytes(P, 1, c->G, c->params.sweep_variant), P.w));
  st = upload_active(c);
  if (st != REWL_OK) return bail(st);
#undef BAIL_CUDA
  *out = c;
  return REWL_OK;
}

void rewl_destroy(rewl_handle h) { delete h; }

static bool with_graph_capture(const rewl_ctx* c) { return c->params.mode == REWL_MODE_GRAPH; }

// One block: sweeps, exchange, clock advance; plus the flatness check when due.
static rewl_status enqueue_block(rewl_ctx* c, bool with_flat) {
  SweepLaunch A{};
  A.n_att = (uint32_t)(c->params.sweeps_per_exchange * c->P.N);
  A.n_active = c->n_active;
  A.wpb = c->wpb;
  A.variant = c->params.sweep_variant;
  A.wait_cycles = c->params.wait_cycles > 0 ? c->params.wait_cycles : kDefaultWaitCycles;
  if (c->pre_on && !with_graph_capture(c)) {
    // this block's draws: prepared by the previous block (checked by its first trial index), else now
    const uint64_t t0 = c->sweep_clock * (uint64_t)c->P.N;
    const int k = c->pre_cur;
    if (c->pre_t0[k] != t0) {
      CUDA_TRY(cudaStreamWaitEvent(c->pre_stream, c->ev_used[k], 0));
      CUDA_TRY(launch_precompute(c->G, c->P, t0, A.n_att, c->pre_stride, c->pre_buf[k], c->n_sm, c->pre_stream));
      CUDA_TRY(cudaEventRecord(c->ev_pre[k], c->pre_stream));
      c->pre_t0[k] = t0;
    }
    CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev_pre[k], 0));
    A.pre = c->pre_buf[k];
    A.pre_stride = c->pre_stride;
  }
  const bool timed = c->params.profile && c->params.mode == REWL_MODE_PLAIN;
  if (timed) {
    if ((int)c->ev_pool.size() < 2 * (c->ev_pending + 1)) {
      cudaEvent_t a, b;
      CUDA_TRY(cudaEventCreate(&a));
      CUDA_TRY(cudaEventCreate(&b));
      c->ev_pool.push_back(a);
      c->ev_pool.push_back(b);
    }
    CUDA_TRY(cudaEventRecord(c->ev_pool[2 * c->ev_pending], c->stream));
  }
  CUDA_TRY(launch_sweep(c->G, c->P, c->S, A, c->stream));
  if (timed) CUDA_TRY(cudaEventRecord(c->ev_pool[2 * c->ev_pending++ + 1], c->stream));
  if (A.pre) {
    // the next block's draws go into the other buffer while this block runs
    const int k = c->pre_cur, k2 = k ^ 1;
    const uint64_t t0n = (c->sweep_clock + (uint64_t)c->params.sweeps_per_exchange) * (uint64_t)c->P.N;
    CUDA_TRY(cudaEventRecord(c->ev_used[k], c->stream));
    CUDA_TRY(cudaStreamWaitEvent(c->pre_stream, c->ev_used[k2], 0));
    CUDA_TRY(launch_precompute(c->G, c->P, t0n, A.n_att, c->pre_stride, c->pre_buf[k2], c->n_sm, c->pre_stream));
    CUDA_TRY(cudaEventRecord(c->ev_pre[k2], c->pre_stream));
    c->pre_t0[k2] = t0n;
    c->pre_cur = k2;
  }
  CUDA_TRY(launch_exchange(c->P, c->S, c->stream));
  CUDA_TRY(launch_advance_clock(c->S, (uint32_t)c->params.sweeps_per_exchange, c->stream));
  if (with_flat) CUDA_TRY(launch_flat_merge(c->P, c->S, c->stream));
  return REWL_OK;
}

// Capture one flatness period (sweeps_per_flat_check / sweeps_per_exchange
// blocks and the flatness check) as a CUDA graph for the current active set.
static rewl_status build_graph(rewl_ctx* c) {
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  const int blocks = c->params.sweeps_per_flat_check / c->params.sweeps_per_exchange;
  cudaGraph_t g;
  CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  rewl_status st = REWL_OK;
  for (int b = 0; b < blocks && st == REWL_OK; ++b) st = enqueue_block(c, b == blocks - 1);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (st != REWL_OK) return st;
  if (e != cudaSuccess) return fail(REWL_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(REWL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  c->graph_n_active = c->n_active;
  return REWL_OK;
}

rewl_status rewl_step(rewl_handle c, int64_t max_sweeps, int32_t* done) {
  if (!c) return fail(REWL_EINVAL, "NULL handle");
  const auto t_start = std::chrono::steady_clock::now();
  const int spe = c->params.sweeps_per_exchange, spf = c->params.sweeps_per_flat_check;
  int64_t swept = 0;
  while (c->n_done < c->P.h && (max_sweeps <= 0 || swept < max_sweeps)) {
    const bool at_boundary = c->sweep_clock % (uint64_t)spf == 0;
    if (c->params.mode == REWL_MODE_GRAPH && at_boundary) {
      if (!c->graph || c->graph_n_active != c->n_active) {
        rewl_status st = build_graph(c);
        if (st != REWL_OK) return st;
      }
      CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
      c->attempts += (uint64_t)c->n_active * (uint64_t)spf * (uint64_t)c->P.N;
      c->sweep_clock += (uint64_t)spf;
      c->xround += (uint64_t)(spf / spe);
      swept += spf;
    } else {
      const bool with_flat = (c->sweep_clock + (uint64_t)spe) % (uint64_t)spf == 0;
      rewl_status st = enqueue_block(c, with_flat);
      if (st != REWL_OK) return st;
      c->attempts += (uint64_t)c->n_active * (uint64_t)spe * (uint64_t)c->P.N;
      c->sweep_clock += (uint64_t)spe;
      c->xround += 1;
      swept += spe;
    }
    if (c->sweep_clock % (uint64_t)spf == 0) {
      CUDA_TRY(d2h(c, c->h_n_done, c->S.n_done, 2 * sizeof(int32_t)));
      CUDA_TRY(cudaStreamSynchronize(c->stream));
      if (c->ev_pending) {
        rewl_status st = collect_sweep_times(c);
        if (st != REWL_OK) return st;
      }
      if (c->h_n_done[1] != 0)
        return fail(REWL_ETIMEOUT, "a sweep kernel's bounded hand-off wait ran out (error bits %d)", c->h_n_done[1]);
      if (*c->h_n_done != c->n_done) {
        rewl_status st = upload_active(c);
        if (st != REWL_OK) return st;
      }
    }
    if (c->params.timeout_ms > 0) {
      const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t_start).count();
      if (ms > c->params.timeout_ms) {
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (done) *done = c->n_done == c->P.h;
        return fail(REWL_ETIMEOUT, "timeout after %lld ms", (long long)ms);
      }
    }
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->ev_pending) {
    rewl_status st = collect_sweep_times(c);
    if (st != REWL_OK) return st;
  }
  if (done) *done = c->n_done == c->P.h;
  return REWL_OK;
}

rewl_status rewl_get_info(rewl_handle c, rewl_info* info) {
  if (!c || !info) return fail(REWL_EINVAL, "NULL argument");
  const Problem& P = c->P;
  info->model = P.model;
  info->q = P.q;
  info->L = P.L;
  info->N = P.N;
  info->windows = P.h;
  info->walkers_per_window = P.m;
  info->window_bins = P.w;
  info->n_bins = P.n_bins;
  info->e_min = P.e_min;
  info->e_max = c->e_max;
  info->e_step = P.e_step;
  info->lattice_words = P.lat_words;
  info->lanes_per_walker = c->G;
  info->walkers_per_block = c->wpb;
  info->mode = c->params.mode;
  info->windows_done = c->n_done;
  info->sweep_clock = (int64_t)c->sweep_clock;
  info->exchange_rounds = (int64_t)c->xround;
  info->attempts = (int64_t)c->attempts;
  info->sweep_launches = c->sweep_launches;
  info->sweep_ms = c->sweep_ms;
  info->h2d_bytes = (int64_t)c->h2d_bytes;
  info->d2h_bytes = (int64_t)c->d2h_bytes;
  info->prefetch_draws = c->pre_on ? 1 : 0;
  info->sweep_variant = c->params.sweep_variant;
  return REWL_OK;
}

rewl_status rewl_get_state(rewl_handle c, rewl_state* st) {
  if (!c || !st) return fail(REWL_EINVAL, "NULL argument");
  const Problem& P = c->P;
  const size_t nW = P.n_walkers;
  cudaStream_t s = c->stream;
  CUDA_TRY(cudaStreamSynchronize(s));
  if (st->lattice) CUDA_TRY(d2h(c, st->lattice, c->S.lat, 4 * nW * P.lat_words));
  if (st->E) CUDA_TRY(d2h(c, st->E, c->S.E, 4 * nW));
  if (st->lng) CUDA_TRY(d2h(c, st->lng, c->S.lng, 8 * nW * P.w));
  if (st->H) CUDA_TRY(d2h(c, st->H, c->S.H, 4 * nW * P.w));
  if (st->win_start) std::memcpy(st->win_start, c->win_start.data(), 4 * P.h);
  if (st->win_width) std::memcpy(st->win_width, c->win_width.data(), 4 * P.h);
  if (st->first_iter) CUDA_TRY(d2h(c, st->first_iter, c->S.first_iter, 8 * P.h));
  if (st->rep_id) CUDA_TRY(d2h(c, st->rep_id, c->S.rep_id, 4 * nW));
  if (st->rep_state) CUDA_TRY(d2h(c, st->rep_state, c->S.rep_state, 4 * nW));
  if (st->rep_trips) CUDA_TRY(d2h(c, st->rep_trips, c->S.rep_trips, 8 * nW));
  if (st->lnf) CUDA_TRY(d2h(c, st->lnf, c->S.lnf, 8 * P.h));
  if (st->iteration) CUDA_TRY(d2h(c, st->iteration, c->S.iter, 4 * P.h));
  if (st->done) CUDA_TRY(d2h(c, st->done, c->S.done, 4 * P.h));
  if (st->stage) CUDA_TRY(d2h(c, st->stage, c->S.stage, 4 * P.h));
  if (st->wl_accept) CUDA_TRY(d2h(c, st->wl_accept, c->S.wl_accept, 8 * nW));
  if (st->near_ties) CUDA_TRY(d2h(c, st->near_ties, c->S.near_ties, 8 * nW));
  if (st->exact_tests) CUDA_TRY(d2h(c, st->exact_tests, c->S.exact_tests, 8 * nW));
  if (st->x_tried) CUDA_TRY(d2h(c, st->x_tried, c->S.x_tried, 8 * P.h));
  if (st->x_accepted) CUDA_TRY(d2h(c, st->x_accepted, c->S.x_accepted, 8 * P.h));
  CUDA_TRY(cudaStreamSynchronize(s));
  st->sweep_clock = (int64_t)c->sweep_clock;
  st->exchange_rounds = (int64_t)c->xround;
  return REWL_OK;
}

rewl_status rewl_set_state(rewl_handle c, const rewl_state* st) {
  if (!c || !st) return fail(REWL_EINVAL, "NULL argument");
  if (!st->lattice || !st->E || !st->lng || !st->H || !st->lnf || !st->iteration || !st->done)
    return fail(REWL_EINVAL, "lattice, E, lng, H, lnf, iteration and done are required");
  if (st->sweep_clock < 0 || st->exchange_rounds < 0 ||
      st->sweep_clock % c->params.sweeps_per_exchange != 0)
    return fail(REWL_EINVAL, "sweep_clock must be a non-negative multiple of sweeps_per_exchange");
  const Problem& P = c->P;
  const size_t nW = P.n_walkers;
  for (int a = 0; a < P.h; ++a)
    if (!is_pow2_double(st->lnf[a]) || st->lnf[a] > 64.0 || (!st->done[a] && st->lnf[a] < 0x1p-39))
      return fail(REWL_EINVAL, "lnf[%d] = %g is not a power of two in [2^-39, 64] (or a finished window's)", a,
                  st->lnf[a]);
  for (size_t W = 0; W < nW; ++W) {
    const int a = (int)(W / P.m);
    const int lo = P.e_min + c->win_start[a] * P.e_step, hi = lo + (c->win_width[a] - 1) * P.e_step;
    if (st->E[W] < lo || st->E[W] > hi || (st->E[W] - P.e_min) % P.e_step) return fail(REWL_EINVAL, "E[%zu] outside its window", W);
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(h2d(c, c->S.lat, st->lattice, 4 * nW * P.lat_words));
  CUDA_TRY(h2d(c, c->S.E, st->E, 4 * nW));
  CUDA_TRY(h2d(c, c->S.lng, st->lng, 8 * nW * P.w));
  CUDA_TRY(h2d(c, c->S.H, st->H, 4 * nW * P.w));
  CUDA_TRY(h2d(c, c->S.lnf, st->lnf, 8 * P.h));
  CUDA_TRY(h2d(c, c->S.iter, st->iteration, 4 * P.h));
  CUDA_TRY(h2d(c, c->S.done, st->done, 4 * P.h));
  if (st->first_iter) CUDA_TRY(h2d(c, c->S.first_iter, st->first_iter, 8 * P.h));
  if (st->rep_id && st->rep_state && st->rep_trips) {
    std::vector<int> seen(nW, 0);
    for (size_t W = 0; W < nW; ++W) {
      if (st->rep_id[W] < 0 || st->rep_id[W] >= (int32_t)nW || seen[st->rep_id[W]]++)
        return fail(REWL_EINVAL, "rep_id is not a permutation of the walkers");
      if (st->rep_state[W] < 0 || st->rep_state[W] > 2) return fail(REWL_EINVAL, "rep_state[%zu]", W);
    }
    CUDA_TRY(h2d(c, c->S.rep_id, st->rep_id, 4 * nW));
    CUDA_TRY(h2d(c, c->S.rep_state, st->rep_state, 4 * nW));
    CUDA_TRY(h2d(c, c->S.rep_trips, st->rep_trips, 8 * nW));
  }
  if (st->stage) {
    for (int a = 0; a < P.h; ++a)
      if (st->stage[a] != 0 && (st->stage[a] != 1 || P.wl_rule != REWL_RULE_ONE_OVER_T))
        return fail(REWL_EINVAL, "stage[%d] = %d", a, st->stage[a]);
    CUDA_TRY(h2d(c, c->S.stage, st->stage, 4 * P.h));
  } else {
    CUDA_TRY(cudaMemsetAsync(c->S.stage, 0, 4 * P.h, c->stream));
  }
  if (st->wl_accept) CUDA_TRY(h2d(c, c->S.wl_accept, st->wl_accept, 8 * nW));
  if (st->near_ties) CUDA_TRY(h2d(c, c->S.near_ties, st->near_ties, 8 * nW));
  if (st->exact_tests) CUDA_TRY(h2d(c, c->S.exact_tests, st->exact_tests, 8 * nW));
  if (st->x_tried) CUDA_TRY(h2d(c, c->S.x_tried, st->x_tried, 8 * P.h));
  if (st->x_accepted) CUDA_TRY(h2d(c, c->S.x_accepted, st->x_accepted, 8 * P.h));
  int nd = 0;
  for (int a = 0; a < P.h; ++a) nd += st->done[a] != 0;
  CUDA_TRY(h2d(c, c->S.n_done, &nd, 4));
  uint64_t clk[2] = {(uint64_t)st->sweep_clock, (uint64_t)st->exchange_rounds};
  CUDA_TRY(h2d(c, c->S.clock, clk, sizeof clk));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->sweep_clock = clk[0];
  c->xround = clk[1];
  return upload_active(c);
}

// Per-window ln g: the mean of the window's m walkers, summed in walker order.
static rewl_status window_means(rewl_ctx* c, std::vector<double>& means) {
  const Problem& P = c->P;
  std::vector<double> lng((size_t)P.n_walkers * P.w);
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  CUDA_TRY(d2h(c, lng.data(), c->S.lng, 8 * lng.size()));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  means.assign((size_t)P.h * P.w, 0.0);
  for (int a = 0; a < P.h; ++a)
    for (int b = 0; b < P.w; ++b) {
      double s = lng[(size_t)(a * P.m) * P.w + b];
      for (int k = 1; k < P.m; ++k) s = s + lng[(size_t)(a * P.m + k) * P.w + b];
      means[(size_t)a * P.w + b] = s / (double)P.m;
    }
  return REWL_OK;
}

rewl_status rewl_get_window_lng(rewl_handle c, int32_t window, int32_t walker, double* lng, int32_t capacity,
                                int32_t* bin_lo, int32_t* n) {
  if (!c || !lng) return fail(REWL_EINVAL, "NULL argument");
  const Problem& P = c->P;
  if (window < 0 || window >= P.h || walker < -1 || walker >= P.m) return fail(REWL_EINVAL, "window/walker index");
  if (capacity < P.w) return fail(REWL_EINVAL, "capacity %d < %d bins", capacity, P.w);
  if (walker >= 0) {
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(d2h(c, lng, c->S.lng + (size_t)(window * P.m + walker) * P.w, 8 * (size_t)P.w));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
  } else {
    std::vector<double> means;
    rewl_status st = window_means(c, means);
    if (st != REWL_OK) return st;
    std::memcpy(lng, means.data() + (size_t)window * P.w, 8 * (size_t)P.w);
  }
  if (bin_lo) *bin_lo = c->win_start[window];
  if (n) *n = c->win_width[window];
  return REWL_OK;
}

// Joining (paper, paragraph after Eq. (1)): window a+1 is shifted onto window
// a at the interior overlap bin where the central differences of ln g -- the
// inverse microcanonical temperatures -- of the two windows agree best (ties
// to the lowest bin); below it window a is kept, above it window a+1.
rewl_status rewl_get_lng(rewl_handle c, double* out, int32_t capacity, int32_t* n_bins, int32_t* e_min,
                         int32_t* e_step) {
  if (!c || !out) return fail(REWL_EINVAL, "NULL argument");
  const Problem& P = c->P;
  if (capacity < P.n_bins) return fail(REWL_EINVAL, "capacity %d < %d bins", capacity, P.n_bins);
  std::vector<double> M;
  rewl_status st = window_means(c, M);
  if (st != REWL_OK) return st;
  const int ld = P.w;  // row stride of the window means; window a has win_width[a] bins
  std::vector<double> g(P.n_bins, -INFINITY);
  for (int b = 0; b < c->win_width[0]; ++b)
    if (M[b] > 0.0) g[c->win_start[0] + b] = M[b];
  double shift_prev = 0.0;
  for (int a = 0; a + 1 < P.h; ++a) {
    const double* A = &M[(size_t)a * ld];
    const double* B = &M[(size_t)(a + 1) * ld];
    const int sa = c->win_start[a], sb = c->win_start[a + 1];
    const int lo = sb, hi = sa + c->win_width[a] - 1;
    int best_b = -1;
    double best = 0.0;
    for (int gb = lo + 1; gb < hi; ++gb) {
      const int ia = gb - sa, ib = gb - sb;
      if (!(A[ia - 1] > 0 && A[ia] > 0 && A[ia + 1] > 0 && B[ib - 1] > 0 && B[ib] > 0 && B[ib + 1] > 0)) continue;
      const double diff = std::fabs((A[ia + 1] - A[ia - 1]) - (B[ib + 1] - B[ib - 1]));
      if (best_b < 0 || diff < best) best = diff, best_b = gb;
    }
    if (best_b < 0)
      for (int gb = lo; gb <= hi; ++gb)
        if (A[gb - sa] > 0 && B[gb - sb] > 0) {
          best_b = gb;
          break;
        }
    if (best_b < 0) return fail(REWL_EINVAL, "windows %d and %d share no visited bin", a, a + 1);
    const double shift = (A[best_b - sa] + shift_prev) - B[best_b - sb];
    for (int gb = best_b + 1; gb < sb + c->win_width[a + 1]; ++gb) {
      const double v = B[gb - sb];
      g[gb] = v > 0 ? v + shift : -INFINITY;
    }
    shift_prev = shift;
  }
  // normalise: sum_E g(E) = q^N
  double mx = -INFINITY;
  for (double v : g) mx = std::max(mx, v);
  if (!std::isfinite(mx)) return fail(REWL_EINVAL, "no visited bin");
  double s = 0.0;
  for (double v : g)
    if (std::isfinite(v)) s += std::exp(v - mx);
  const double shift = (double)P.N * std::log((double)P.q) - (mx + std::log(s));
  for (int b = 0; b < P.n_bins; ++b) out[b] = std::isfinite(g[b]) ? g[b] + shift : -INFINITY;
  if (n_bins) *n_bins = P.n_bins;
  if (e_min) *e_min = P.e_min;
  if (e_step) *e_step = P.e_step;
  return REWL_OK;
}


// Run-time balanced partition (Fig. 1b and the speed-up paragraph: windows
// sized so that every window finishes its first iteration after the same
// number of sweeps, estimated from a pre-run with equal windows).  Reading:
// the first iteration of a window is a diffusive walk whose duration is
// (sum over its bins of rho(b))^2; pre-run window a (first merge after tau_a
// sweeps, width w_a) gives rho_a = sqrt(tau_a) / w_a, and rho(b) is the mean
// of rho_a over the pre-run windows containing b.  With U(b) = rho(0) + ... +
// rho(b-1), the new windows are the equal partition of Fig. 1a laid out in U:
// length lam = U(B) / (1 + (h-1)(1-o)), window k covers [u_k, u_k + lam],
// u_k = k (U(B) - lam) / (h-1); it starts at the last bin b with U(b) <= u_k
// and ends at the first bin b with U(b+1) >= u_k + lam (the first window at
// bin 0, the last at bin B-1).
rewl_status rewl_plan_windows(const int64_t* first_iter_sweeps, const int32_t* pre_starts, const int32_t* pre_widths,
                              int32_t pre_windows, int32_t n_bins, int32_t windows, double overlap, int32_t* starts,
                              int32_t* widths) {
  if (!first_iter_sweeps || !pre_starts || !pre_widths || !starts || !widths || pre_windows < 1 || n_bins < 3 ||
      windows < 1 || !(overlap > 0.0 && overlap < 1.0))
    return fail(REWL_EINVAL, "rewl_plan_windows: invalid argument");
  rewl_status st = check_windows(n_bins, pre_windows, pre_starts, pre_widths);
  if (st != REWL_OK) return st;
  std::vector<double> rho_w(pre_windows);
  for (int a = 0; a < pre_windows; ++a) {
    if (first_iter_sweeps[a] <= 0) return fail(REWL_EINVAL, "window %d has not finished its first iteration", a);
    rho_w[a] = std::sqrt((double)first_iter_sweeps[a]) / (double)pre_widths[a];
  }
  std::vector<double> U(n_bins + 1, 0.0);
  for (int b = 0; b < n_bins; ++b) {
    double sum = 0.0;
    int n = 0;
    for (int a = 0; a < pre_windows; ++a)
      if (pre_starts[a] <= b && b < pre_starts[a] + pre_widths[a]) {
        sum = sum + rho_w[a];
        ++n;
      }
    U[b + 1] = U[b] + sum / (double)n;
  }
  if (windows == 1) {
    starts[0] = 0;
    widths[0] = n_bins;
    return REWL_OK;
  }
  const double T = U[n_bins];
  const double lam = T / (1.0 + (double)(windows - 1) * (1.0 - overlap));
  std::vector<int32_t> s0(windows), w0(windows);
  for (int k = 0; k < windows; ++k) {
    const double u_lo = ((double)k * (T - lam)) / (double)(windows - 1);
    const double u_hi = u_lo + lam;
    int first = 0, last = n_bins - 1;
    if (k > 0)
      for (int b = 0; b < n_bins; ++b)
        if (U[b] <= u_lo) first = b;
    if (k < windows - 1)
      for (int b = 0; b < n_bins; ++b)
        if (U[b + 1] >= u_hi) {
          last = b;
          break;
        }
    s0[k] = first;
    w0[k] = last - first + 1;
  }
  st = check_windows(n_bins, windows, s0.data(), w0.data());
  if (st != REWL_OK) return st;
  std::memcpy(starts, s0.data(), sizeof(int32_t) * windows);
  std::memcpy(widths, w0.data(), sizeof(int32_t) * windows);
  return REWL_OK;
}

}  // extern "C"
