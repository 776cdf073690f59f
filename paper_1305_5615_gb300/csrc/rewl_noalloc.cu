// rewl_noalloc.cu -- rewl_sweep_noalloc: the WL sweep kernel run on state the
// caller keeps in its own device memory, with every piece of working memory
// the kernel needs beyond that state taken from one fixed array compiled into
// the library.  The call itself allocates nothing.
//
// Some callers cannot allocate device memory at the time they want to run a
// sweep: code that runs inside a memory pool or arena it does not control,
// an embedding runtime whose allocator must not be re-entered from a library
// call, or a process that has reserved all device memory up front.  They own
// the state buffers already and only need the kernel.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "rewl.h"
#include "rewl_kernels.h"
#include "rewl_layout.h"

using namespace rewl;

namespace {

// Working memory of one call, shared by all calls on a device:
//   [0, 16)                       sweep clock (u64) and exchange round (u64)
//   then, each for REWL_NOALLOC_MAX_WALKERS walkers:
//   active walker ids (i32), status flags (i32), accepted moves, near ties and
//   exact tests (u64 each).
constexpr size_t kClockBytes = 16;
constexpr size_t kMaxW = REWL_NOALLOC_MAX_WALKERS;
constexpr size_t kScratchBytes = kClockBytes + kMaxW * (4 + 4 + 8 + 8 + 8);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device (the host-side name of the array is only a stand-in) and kept
// for the life of the process (it belongs to the device's primary context).
rewl_status scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return REWL_ENODEV;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return REWL_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return REWL_OK;
}

// Clears the part of the scratch a call uses (and the caller's status array,
// when given: S.status points there) and fills the walker list; the sweep
// kernel marks the walkers it skips (E outside the window, ln f not usable).
__global__ void k_noalloc_prepare(DevState S, int n_walkers, uint64_t first_sweep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    S.clock[0] = first_sweep;
    S.clock[1] = 0;
  }
  if (i < n_walkers) {
    S.active[i] = i;
    S.status[i] = 0;
    S.wl_accept[i] = 0;
    S.near_ties[i] = 0;
    S.exact_tests[i] = 0;
  }
}

}  // namespace

void rewl_set_last_error(const char* msg);

extern "C" rewl_status rewl_sweep_noalloc(const rewl_sweep_desc* d, uint32_t* lattice, int32_t* E, double* lng,
                                          uint32_t* H, const uint32_t* coupling_bits, const int32_t* win_start,
                                          const double* lnf, void* stream) {
  if (!d || !lattice || !E || !lng || !H || !win_start || !lnf) {
    rewl_set_last_error("rewl_sweep_noalloc: NULL argument");
    return REWL_EINVAL;
  }
  const int L = d->L;
  const int64_t n_walkers = (int64_t)d->windows * d->walkers_per_window;
  if (d->model < 0 || d->model > 2 || L < 2 || L > 256 || d->windows < 1 || d->walkers_per_window < 1 ||
      d->window_bins < 3 || d->e_step < 1 || d->sweeps < 0 || (d->model == REWL_POTTS && (d->q < 2 || d->q > 16)) ||
      (d->model == REWL_EA_PM_J && !coupling_bits)) {
    rewl_set_last_error("rewl_sweep_noalloc: invalid descriptor");
    return REWL_EINVAL;
  }
  if (n_walkers > (int64_t)kMaxW) {
    rewl_set_last_error("rewl_sweep_noalloc: more walkers than REWL_NOALLOC_MAX_WALKERS (4096)");
    return REWL_EINVAL;
  }
  if ((int64_t)d->sweeps * L * L > 0x7fffffffLL) {
    rewl_set_last_error("rewl_sweep_noalloc: sweeps * L * L exceeds 2^31 - 1 trials per walker");
    return REWL_EINVAL;
  }
  const int G = d->lanes_per_walker ? d->lanes_per_walker : 32;
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32) {
    rewl_set_last_error("rewl_sweep_noalloc: lanes_per_walker must be 1, 2, 4, 8, 16 or 32");
    return REWL_EINVAL;
  }
  unsigned char* base = nullptr;
  rewl_status st = scratch_address(&base);
  if (st != REWL_OK) {
    rewl_set_last_error("rewl_sweep_noalloc: cannot resolve the device address of the scratch array");
    return st;
  }
  Problem P{};
  P.model = d->model;
  P.q = d->model == REWL_POTTS ? d->q : 2;
  P.L = L;
  P.N = L * L;
  P.Wr = d->model == REWL_POTTS ? (L + 7) / 8 : (L + 31) / 32;
  P.Wr1 = (L + 31) / 32;
  P.rows = L;
  P.lat_words = L * P.Wr;
  P.j_words = 2 * L * P.Wr1;
  P.e_min = d->e_min;
  P.e_step = d->e_step;
  P.h = d->windows;
  P.m = d->walkers_per_window;
  P.w = d->window_bins;
  P.n_walkers = (int)n_walkers;
  P.n_bins = 0;
  P.magic_L = (uint32_t)(((1ull << 32) + (uint64_t)L - 1) / (uint64_t)L);
  P.seed_lo = (uint32_t)d->seed;
  P.seed_hi = (uint32_t)(d->seed >> 32);
  DevState S{};
  S.lat = lattice;
  S.J = const_cast<uint32_t*>(coupling_bits);
  S.E = E;
  S.lng = lng;
  S.H = H;
  S.win_start = const_cast<int32_t*>(win_start);
  S.lnf = const_cast<double*>(lnf);
  S.clock = reinterpret_cast<uint64_t*>(base);
  unsigned char* q = base + kClockBytes;
  S.active = reinterpret_cast<int32_t*>(q);
  q += kMaxW * 4;
  S.status = d->status ? d->status : reinterpret_cast<int32_t*>(q);  // the caller's array, if given
  q += kMaxW * 4;
  S.wl_accept = reinterpret_cast<uint64_t*>(q);
  q += kMaxW * 8;
  S.near_ties = reinterpret_cast<uint64_t*>(q);
  q += kMaxW * 8;
  S.exact_tests = reinterpret_cast<uint64_t*>(q);

  const int wpb = 1;
  if (sweep_smem_bytes(P, wpb, G, kSweepChain) > 227 * 1024) {
    rewl_set_last_error("rewl_sweep_noalloc: one walker's window does not fit in shared memory");
    return REWL_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prepare_sweep(G, P.model) != cudaSuccess) {
    rewl_set_last_error("rewl_sweep_noalloc: cudaFuncSetAttribute failed");
    return REWL_ECUDA;
  }
  k_noalloc_prepare<<<(int)((n_walkers + 127) / 128), 128, 0, s>>>(S, (int)n_walkers, d->first_sweep);
  if (cudaGetLastError() != cudaSuccess) {
    rewl_set_last_error("rewl_sweep_noalloc: launch failed");
    return REWL_ECUDA;
  }
  if (d->sweeps == 0) return REWL_OK;
  SweepLaunch A{};
  A.n_att = (uint32_t)(d->sweeps * P.N);
  A.n_active = (int)n_walkers;
  A.wpb = wpb;
  A.variant = kSweepChain;
  if (launch_sweep(G, P, S, A, s) != cudaSuccess) {
    rewl_set_last_error("rewl_sweep_noalloc: sweep launch failed");
    return REWL_ECUDA;
  }
  return REWL_OK;
}
