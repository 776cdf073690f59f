// rates.cu -- microbenchmarks of the GB300 rates that bound the REWL sweep
// kernel: integer issue rates of the operation mixes one trial needs (the
// Philox round's 32x32->64 multiply with a three-input XOR; the 32-bit
// multiply, add and XOR), FP64 add throughput and latency, double log and float logf
// throughput, Philox4x32-10 throughput (the library's own generator),
// shared-memory load and warp-shuffle latency, and the latency of the
// sequential WL step itself (the chain bin -> shadow loads -> 64-bit compare
// -> next bin) stripped of everything the sweep kernel does around it.
//
// Throughputs are per SM per clock: every block measures its own clock64
// interval, all blocks of a launch are resident at once, and
//   rate = (operations of the blocks on one SM) / (median block cycles).
// Latencies are cycles per step of one dependent chain in one thread.
//
// Build and run: python -m ubench
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "rewl_device.cuh"

#define CK(x)                                                                      \
  do {                                                                             \
    cudaError_t e_ = (x);                                                          \
    if (e_ != cudaSuccess) {                                                       \
      std::fprintf(stderr, "%s:%d %s\n", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return 1;                                                                    \
    }                                                                              \
  } while (0)

namespace {

__device__ __forceinline__ void stamp(long long* cyc, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) cyc[blockIdx.x] = clock64() - t0;
}

// ---- integer mixes, 8 independent chains per thread; each step is two lane
// operations as written (a multiply or a three-input add, then a three-input
// XOR that feeds the next step), so nothing can be folded away:
//   MIX 0: t = a * M (32 x 32 -> 64); a = hi(t) ^ b ^ k; b = lo(t)  -- half a Philox round
//   MIX 1: a = (a * M) ^ b ^ k (low 32 bits); b = a + b               -- 32-bit multiply, add
//   MIX 2: a = a + b + k; b = a ^ b ^ k                              -- add and XOR only
template <int MIX>
__global__ void k_int_tput(uint32_t* out, long long* cyc, int iters) {
  uint32_t a[8], b[8];
  for (int q = 0; q < 8; ++q) {
    a[q] = threadIdx.x * 0x9E3779B9u + q;
    b[q] = blockIdx.x + 0x7F4A7C15u * q;
  }
  const uint32_t k = 0xBB67AE85u ^ blockIdx.x, M = 0xD2511F53u;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if constexpr (MIX == 0) {
        const uint64_t t = (uint64_t)a[q] * M;
        a[q] = (uint32_t)(t >> 32) ^ b[q] ^ k;
        b[q] = (uint32_t)t;
      } else if constexpr (MIX == 1) {
        a[q] = (a[q] * M) ^ b[q] ^ k;
        b[q] = a[q] + b[q];
      } else {
        a[q] = a[q] + b[q] + k;
        b[q] = a[q] ^ b[q] ^ k;
      }
    }
  }
  stamp(cyc, t0);
  uint32_t s = 0;
  for (int q = 0; q < 8; ++q) s ^= a[q] + b[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---- FP64 add: 8 independent chains per thread
__global__ void k_dadd_tput(double* out, long long* cyc, int iters) {
  double a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
  const double c = 1e-9 * (blockIdx.x + 1);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a[k] + c;
  stamp(cyc, t0);
  double s = 0;
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---- FP64 add: one dependent chain
__global__ void k_dadd_lat(double* out, long long* cyc, int iters) {
  double a = threadIdx.x;
  const double c = 1e-9;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) a = a + c;
  cyc[0] = clock64() - t0;
  out[0] = a;
}

// ---- double log / float logf on independent arguments
__global__ void k_log_tput(double* out, long long* cyc, int iters) {
  double x = 1.0 + 1e-3 * threadIdx.x, s = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    s += log(x);
    x += 0.5;
  }
  stamp(cyc, t0);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_logf_tput(float* out, long long* cyc, int iters) {
  float x0 = 1.0f + 1e-3f * threadIdx.x, x1 = x0 + 0.25f, x2 = x0 + 0.5f, x3 = x0 + 0.75f;
  float s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    s0 += logf(x0);
    s1 += logf(x1);
    s2 += logf(x2);
    s3 += logf(x3);
    x0 += 1.0f;
    x1 += 1.0f;
    x2 += 1.0f;
    x3 += 1.0f;
  }
  stamp(cyc, t0);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s0 + s1 + s2 + s3;
}

// ---- Philox4x32-10, the library's definition
__global__ void k_philox_tput(uint32_t* out, long long* cyc, int iters) {
  const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
    const rewl::U4 r = rewl::philox10((uint32_t)i, 0u, id, 0u, 0x12345678u, 0x9abcdef0u);
    acc ^= r.x ^ r.y ^ r.z ^ r.w;
  }
  stamp(cyc, t0);
  out[id] = acc;
}

// ---- shared-memory load latency: pointer chase over a random cycle of 1024 words
__global__ void k_lds_lat(int* out, long long* cyc, int iters) {
  __shared__ int nxt[1024];
  if (threadIdx.x == 0) {  // one cycle through all 1024 slots, stride 97 (odd, so a single cycle)
    for (int i = 0; i < 1024; ++i) nxt[i] = (i + 97) & 1023;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int p = 0;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) p = nxt[p];
  cyc[0] = clock64() - t0;
  out[0] = p;
}

// ---- warp shuffle latency: a value passed around the warp
__global__ void k_shfl_lat(int* out, long long* cyc, int iters) {
  int v = threadIdx.x;
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) v = __shfl_sync(0xffffffffu, v, (threadIdx.x + 1) & 31) + 1;
  if (threadIdx.x == 0) {
    cyc[0] = clock64() - t0;
    out[0] = v;
  }
}

// ---- the sequential WL step on its own.  One walker per block (lane 0), a
// window of W bins whose int64 shadow lives in shared memory with 4 guard
// bins on each side, bin offsets in -2..2 and thresholds ln u * 2^40 made
// beforehand.  variant 0: the dependency chain only (two candidate loads for
// the next trial, the compare, the write-back of the bin left, the selects);
// variant 1: plus the guard-band and conflict tests folded into a flag;
// variant 2: the tests as a branch out of the loop (never taken here), as
// the sweep kernel has them.  T = long long is the fixed-point shadow the
// sweep kernel uses (units of 2^-40); T = double is the same step on FP64
// ln g values, for comparison.
constexpr int kSteps = 2048;  // inputs per pass, reused cyclically
constexpr int kMaxW = 512;

template <typename T>
__device__ __forceinline__ T fx_scale(double v) {
  if constexpr (sizeof(T) == 8 && T(0.5) == T(0)) return (T)(v * 1099511627776.0);
  else return (T)v;
}

template <int VARIANT, typename T = long long>
__global__ void k_chain(int W, int passes, long long* cyc, long long* out) {
  __shared__ int s_d[kSteps];
  __shared__ T s_thr[kSteps];
  __shared__ unsigned s_mask[kSteps];
  __shared__ T s_fx[kMaxW + 8];
  for (int i = threadIdx.x; i < kSteps; i += blockDim.x) {
    const rewl::U4 r = rewl::philox10((uint32_t)i, blockIdx.x, 7u, 0u, 0x2468aceu, 0x13579bdu);
    const uint32_t k = rewl::scale32(r.x, 16u);  // 0, +-1 often; +-2 rarely (a 2D Ising walk's mix)
    s_d[i] = k < 6 ? 0 : k < 10 ? 1 : k < 14 ? -1 : k < 15 ? 2 : -2;
    const float u = ((float)(r.y >> 8) + 0.5f) * 0x1p-24f;
    s_thr[i] = fx_scale<T>((double)logf(u));
    s_mask[i] = 0u;
  }
  for (int b = threadIdx.x; b < W + 8; b += blockDim.x) {  // a smooth ln g-like shadow
    const double x = (double)(b - 4) / W;
    s_fx[b] = fx_scale<T>(200.0 * x * (1.0 - x) + 1.0);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  T* fxp = s_fx + 4;
  const T lnf = fx_scale<T>(0x1p-10), guard = fx_scale<T>(0x1p-16);
  int bin = W / 2, d = s_d[0];
  T fx_cur = fxp[bin], fxn = fxp[bin + d];
  unsigned accm = 0, bad = 0;
  const long long t0 = clock64();
  for (int p = 0; p < passes; ++p) {
#pragma unroll 1
    for (int j = 0; j < kSteps; ++j) {
      const int dn = s_d[(j + 1) & (kSteps - 1)];
      const T thr = s_thr[j];
      const int bn = bin + d;
      const T cs = fxp[bin + dn], cm = fxp[bn + dn];
      const bool inwin = (unsigned)bn < (unsigned)W;
      const T lim_acc = fx_cur - thr - guard;
      const bool acc = d == 0 || (inwin && fxn < lim_acc);
      if (VARIANT >= 1) {
        const T lim_rej = fx_cur - thr + guard;
        const bool band = d != 0 && inwin && fxn >= lim_acc && fxn <= lim_rej;
        const bool hit = band || (accm & s_mask[j]) != 0u;
        if (VARIANT == 2) {
          if (hit) {  // never taken: no conflicts are planted and the band is 3e-5 wide
            bad += 1u + (unsigned)j;
            break;
          }
        } else {
          bad |= (unsigned)hit;
        }
        accm = (accm << 1) | (unsigned)acc;
      }
      const bool mv = acc && d != 0;
      if (mv) fxp[bin] = fx_cur;
      const T fwd = (dn == -d) ? fx_cur : cm;
      fx_cur = (mv ? fxn : fx_cur) + lnf;
      fxn = mv ? fwd : cs;
      bin = mv ? bn : bin;
      d = dn;
    }
  }
  cyc[blockIdx.x] = clock64() - t0;
  out[blockIdx.x] = (long long)fx_cur + bin + bad;
}

// The same step with trial j+1's test made for both outcomes of trial j
// before that outcome is known (the outcome then only selects between two
// ready predicates): a candidate restructuring of the sweep kernel's fast
// loop, measured here on its own.  Inputs and results as k_chain<0>.
__global__ void k_chain_spec(int W, int passes, long long* cyc, long long* out) {
  __shared__ int s_d[kSteps];
  __shared__ long long s_thr[kSteps];
  __shared__ long long s_fx[kMaxW + 8];
  for (int i = threadIdx.x; i < kSteps; i += blockDim.x) {
    const rewl::U4 r = rewl::philox10((uint32_t)i, blockIdx.x, 7u, 0u, 0x2468aceu, 0x13579bdu);
    const uint32_t k = rewl::scale32(r.x, 16u);
    s_d[i] = k < 6 ? 0 : k < 10 ? 1 : k < 14 ? -1 : k < 15 ? 2 : -2;
    const float u = ((float)(r.y >> 8) + 0.5f) * 0x1p-24f;
    s_thr[i] = fx_scale<long long>((double)logf(u));
  }
  for (int b = threadIdx.x; b < W + 8; b += blockDim.x) {
    const double x = (double)(b - 4) / W;
    s_fx[b] = fx_scale<long long>(200.0 * x * (1.0 - x) + 1.0);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  long long* fxp = s_fx + 4;
  const long long lnf = 1ll << 30, guard = 1ll << 24;
  int bin = W / 2, d = s_d[0];
  long long fx_cur = fxp[bin], fxn = fxp[bin + d];
  bool A = d == 0 || ((unsigned)(bin + d) < (unsigned)W && fxn < fx_cur - s_thr[0] - guard);
  const long long t0 = clock64();
  for (int p = 0; p < passes; ++p) {
#pragma unroll 1
    for (int j = 0; j < kSteps; ++j) {
      const int j1 = (j + 1) & (kSteps - 1);
      const int dn = s_d[j1];
      const long long thr1 = s_thr[j1] + guard;
      const int bn = bin + d;
      const long long cs = fxp[bin + dn], cm = fxp[bn + dn];
      const bool mv = A && d != 0;
      if (mv) fxp[bin] = fx_cur;
      const long long fwd = (dn == -d) ? fx_cur : cm;
      const long long fcs = fx_cur + lnf, fcm = fxn + lnf;
      const bool As = dn == 0 || ((unsigned)(bin + dn) < (unsigned)W && cs < fcs - thr1);
      const bool Am = dn == 0 || ((unsigned)(bn + dn) < (unsigned)W && fwd < fcm - thr1);
      A = mv ? Am : As;
      fxn = mv ? fwd : cs;
      fx_cur = mv ? fcm : fcs;
      bin = mv ? bn : bin;
      d = dn;
    }
  }
  cyc[blockIdx.x] = clock64() - t0;
  out[blockIdx.x] = fx_cur + bin;
}

// The same step with the candidate shadows loaded one trial further ahead:
// in the iteration of trial j the shadows trial j+2 may target are loaded
// for all four outcomes of trials j and j+1; the next iteration keeps the
// two that trial j's outcome allows (with trial j's write-back forwarded).
// A load then has a whole iteration to arrive instead of part of one.
// Inputs and results as k_chain<0>.
__global__ void k_chain_deep3(int W, int passes, long long* cyc, long long* out) {
  __shared__ int s_d[kSteps];
  __shared__ long long s_thr[kSteps];
  __shared__ long long s_fx[kMaxW + 16];
  for (int i = threadIdx.x; i < kSteps; i += blockDim.x) {
    const rewl::U4 r = rewl::philox10((uint32_t)i, blockIdx.x, 7u, 0u, 0x2468aceu, 0x13579bdu);
    const uint32_t k = rewl::scale32(r.x, 16u);
    s_d[i] = k < 6 ? 0 : k < 10 ? 1 : k < 14 ? -1 : k < 15 ? 2 : -2;
    const float u = ((float)(r.y >> 8) + 0.5f) * 0x1p-24f;
    s_thr[i] = fx_scale<long long>((double)logf(u));
  }
  for (int b = threadIdx.x; b < W + 16; b += blockDim.x) {  // the same shadow as k_chain, 8 guard bins
    const double x = (double)(b - 8) / W;
    s_fx[b] = fx_scale<long long>(200.0 * x * (1.0 - x) + 1.0);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  long long* fxp = s_fx + 8;  // bins -8 .. W+7; loads reach B + 3 offsets of at most 2
  const long long lnf = 1ll << 30, guard = 1ll << 24;
  int B = W / 2;
  long long X = fxp[B], Y = fxp[B + s_d[0]];
  long long Rss = fxp[B + s_d[1]], Rsm = fxp[B + s_d[0] + s_d[1]], Rms = Rss, Rmm = Rsm;
  bool mvp = false;
  int Bp = B;
  long long Xp = X;
  const long long t0 = clock64();
  for (int p = 0; p < passes; ++p) {
#pragma unroll 1
    for (int j = 0; j < kSteps; ++j) {
      const int dj = s_d[j], d1 = s_d[(j + 1) & (kSteps - 1)], d2 = s_d[(j + 2) & (kSteps - 1)];
      const long long thr = s_thr[j];
      // loads for trial j+2 (memory holds every write-back up to trial j-1)
      const long long nss = fxp[B + d2], nsm = fxp[B + d1 + d2], nms = fxp[B + dj + d2], nmm = fxp[B + dj + d1 + d2];
      // trial j+1's candidates from the loads of the last iteration
      const int Ts = B + d1, Tm = B + dj + d1;
      long long Cs = mvp ? Rms : Rss, Cm = mvp ? Rmm : Rsm;
      if (mvp && Ts == Bp) Cs = Xp;
      if (mvp && Tm == Bp) Cm = Xp;
      // trial j
      const int bn = B + dj;
      const bool acc = dj == 0 || ((unsigned)bn < (unsigned)W && Y < X - thr - guard);
      const bool mv = acc && dj != 0;
      if (mv) fxp[B] = X;
      const long long Yn = mv ? (d1 == -dj ? X : Cm) : Cs;
      const long long Xn = (mv ? Y : X) + lnf;
      mvp = mv;
      Bp = B;
      Xp = X;
      Rss = nss;
      Rsm = nsm;
      Rms = nms;
      Rmm = nmm;
      B = mv ? bn : B;
      X = Xn;
      Y = Yn;
    }
  }
  cyc[blockIdx.x] = clock64() - t0;
  out[blockIdx.x] = X + B;
}

// The step with the band and conflict tests of two trials folded into one
// branch: trial j+1 is evaluated from trial j's outcome as if trial j needed
// no slow path, its write-back is predicated on neither needing it, and the
// loop leaves (for the slow path; never taken here but on the rare band case)
// once per pair.  Inputs as k_chain<1>.
__global__ void k_chain_pair(int W, int passes, long long* cyc, long long* out) {
  __shared__ int s_d[kSteps];
  __shared__ long long s_thr[kSteps];
  __shared__ unsigned s_mask[kSteps];
  __shared__ long long s_fx[kMaxW + 8];
  for (int i = threadIdx.x; i < kSteps; i += blockDim.x) {
    const rewl::U4 r = rewl::philox10((uint32_t)i, blockIdx.x, 7u, 0u, 0x2468aceu, 0x13579bdu);
    const uint32_t k = rewl::scale32(r.x, 16u);
    s_d[i] = k < 6 ? 0 : k < 10 ? 1 : k < 14 ? -1 : k < 15 ? 2 : -2;
    const float u = ((float)(r.y >> 8) + 0.5f) * 0x1p-24f;
    s_thr[i] = fx_scale<long long>((double)logf(u));
    s_mask[i] = 0u;
  }
  for (int b = threadIdx.x; b < W + 8; b += blockDim.x) {
    const double x = (double)(b - 4) / W;
    s_fx[b] = fx_scale<long long>(200.0 * x * (1.0 - x) + 1.0);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  long long* fxp = s_fx + 4;
  const long long lnf = 1ll << 30, guard = 1ll << 24;
  int bin = W / 2, d = s_d[0];
  long long fx_cur = fxp[bin], fxn = fxp[bin + d];
  unsigned accm = 0, bad = 0;
  const long long t0 = clock64();
  for (int p = 0; p < passes; ++p) {
#pragma unroll 1
    for (int j = 0; j < kSteps; j += 2) {
      const int d1 = s_d[j + 1], d2 = s_d[(j + 2) & (kSteps - 1)];
      const long long thr0 = s_thr[j], thr1 = s_thr[j + 1];
      const unsigned m0 = s_mask[j], m1 = s_mask[j + 1];
      // trial j
      const int bn = bin + d;
      const long long cs = fxp[bin + d1], cm = fxp[bn + d1];
      const bool in0 = (unsigned)bn < (unsigned)W;
      const long long la0 = fx_cur - thr0 - guard, lr0 = fx_cur - thr0 + guard;
      const bool acc0 = d == 0 || (in0 && fxn < la0);
      const bool hit0 = (d != 0 && in0 && fxn >= la0 && fxn <= lr0) || (accm & m0) != 0u;
      const bool mv0 = acc0 && d != 0;
      if (mv0 && !hit0) fxp[bin] = fx_cur;
      const long long fwd0 = (d1 == -d) ? fx_cur : cm;
      const long long x1 = (mv0 ? fxn : fx_cur) + lnf, y1 = mv0 ? fwd0 : cs;
      const int b1 = mv0 ? bn : bin;
      const unsigned accm1 = (accm << 1) | (unsigned)acc0;
      // trial j+1, as if trial j needed no slow path
      const int bn1 = b1 + d1;
      const long long cs1 = fxp[b1 + d2], cm1 = fxp[bn1 + d2];
      const bool in1 = (unsigned)bn1 < (unsigned)W;
      const long long la1 = x1 - thr1 - guard, lr1 = x1 - thr1 + guard;
      const bool acc1 = d1 == 0 || (in1 && y1 < la1);
      const bool hit1 = (d1 != 0 && in1 && y1 >= la1 && y1 <= lr1) || (accm1 & m1) != 0u;
      const bool mv1 = acc1 && d1 != 0;
      if (mv1 && !hit0 && !hit1) fxp[b1] = x1;
      if (hit0 || hit1) {  // the slow path would take over here
        bad += 1u + (unsigned)j;
        break;
      }
      const long long fwd1 = (d2 == -d1) ? x1 : cm1;
      fx_cur = (mv1 ? y1 : x1) + lnf;
      fxn = mv1 ? fwd1 : cs1;
      bin = mv1 ? bn1 : b1;
      accm = (accm1 << 1) | (unsigned)acc1;
      d = d2;
    }
  }
  cyc[blockIdx.x] = clock64() - t0;
  out[blockIdx.x] = fx_cur + bin + bad;
}

double median(std::vector<long long> v) {
  std::sort(v.begin(), v.end());
  return (double)v[v.size() / 2];
}

}  // namespace

int main() {
  int dev = 0, n_sm = 0, khz = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  std::printf("device SMs %d, max SM clock %.0f MHz\n", n_sm, khz / 1e3);
  const int bps = 4, threads = 256, blocks = n_sm * bps;  // 1024 threads per SM, all resident
  double* d_out = nullptr;
  long long* d_cyc = nullptr;
  CK(cudaMalloc(&d_out, sizeof(double) * blocks * threads));
  CK(cudaMalloc(&d_cyc, sizeof(long long) * blocks));
  std::vector<long long> cyc(blocks);
  auto per_sm_clk = [&](double ops_per_block) {
    cudaMemcpy(cyc.data(), d_cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
    return ops_per_block * bps / median(cyc);
  };
  long long one = 0;

  const char* mix_names[3] = {"32x32->64 multiply + XOR3 (Philox round mix)", "32-bit multiply + XOR3, add",
                              "add3 + XOR3"};
  const int it_int = 1 << 12;
  for (int mix = 0; mix < 3; ++mix) {
    uint32_t* o = reinterpret_cast<uint32_t*>(d_out);
    if (mix == 0) k_int_tput<0><<<blocks, threads>>>(o, d_cyc, 16);
    if (mix == 0) k_int_tput<0><<<blocks, threads>>>(o, d_cyc, it_int);
    if (mix == 1) k_int_tput<1><<<blocks, threads>>>(o, d_cyc, it_int);
    if (mix == 2) k_int_tput<2><<<blocks, threads>>>(o, d_cyc, it_int);
    CK(cudaDeviceSynchronize());
    std::printf("integer mix %d, %-46s %8.2f lane-ops/clk/SM\n", mix, mix_names[mix],
                per_sm_clk((double)threads * 8 * 2 * it_int));
  }

  const int it_add = 1 << 14;
  k_dadd_tput<<<blocks, threads>>>(d_out, d_cyc, 16);
  k_dadd_tput<<<blocks, threads>>>(d_out, d_cyc, it_add);
  CK(cudaDeviceSynchronize());
  std::printf("FP64 add, 8 independent chains per thread:  %8.3f lane-ops/clk/SM\n",
              per_sm_clk((double)threads * 8 * it_add));
  k_dadd_lat<<<1, 1>>>(d_out, d_cyc, 1 << 14);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&one, d_cyc, sizeof(long long), cudaMemcpyDeviceToHost));
  std::printf("FP64 add dependent latency:                 %8.1f clk\n", (double)one / (1 << 14));

  const int it_log = 1 << 9;
  k_log_tput<<<blocks, threads>>>(d_out, d_cyc, it_log);
  CK(cudaDeviceSynchronize());
  std::printf("double log():                               %8.3f lane-ops/clk/SM\n",
              per_sm_clk((double)threads * it_log));
  const int it_logf = 1 << 12;
  k_logf_tput<<<blocks, threads>>>(reinterpret_cast<float*>(d_out), d_cyc, it_logf);
  CK(cudaDeviceSynchronize());
  std::printf("float logf():                               %8.2f lane-ops/clk/SM\n",
              per_sm_clk((double)threads * 4 * it_logf));
  const int it_ph = 1 << 11;
  k_philox_tput<<<blocks, threads>>>(reinterpret_cast<uint32_t*>(d_out), d_cyc, it_ph);
  CK(cudaDeviceSynchronize());
  const double ph = per_sm_clk((double)threads * it_ph);
  std::printf("Philox4x32-10 (10 rounds):                  %8.3f calls/clk/SM (%.2e calls/s at the max clock)\n",
              ph, ph * n_sm * khz * 1e3);

  k_lds_lat<<<1, 32>>>(reinterpret_cast<int*>(d_out), d_cyc, 1 << 14);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&one, d_cyc, sizeof(long long), cudaMemcpyDeviceToHost));
  std::printf("shared-memory load dependent latency:       %8.1f clk\n", (double)one / (1 << 14));
  k_shfl_lat<<<1, 32>>>(reinterpret_cast<int*>(d_out), d_cyc, 1 << 14);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&one, d_cyc, sizeof(long long), cudaMemcpyDeviceToHost));
  std::printf("warp shuffle (+1) dependent latency:        %8.1f clk\n", (double)one / (1 << 14));

  // the sequential WL step: 64 walkers on 64 SMs, window of 216 bins (Ising 32x32, 16 windows)
  const int W = 216, passes = 64, nb = 64;
  const char* names[8] = {"dependency chain only", "+ band and conflict tests as a flag",
                          "+ the tests as a branch out of the loop", "FP64 ln g, dependency chain only",
                          "FP64 ln g, + the tests as a branch", "next test made for both outcomes",
                          "candidate loads a trial further ahead", "+ the tests as one branch per pair"};
  std::vector<long long> ref;
  for (int v = 0; v < 8; ++v) {
    long long* o = reinterpret_cast<long long*>(d_out);
    if (v == 0) k_chain<0><<<nb, 32>>>(W, passes, d_cyc, o);
    if (v == 1) k_chain<1><<<nb, 32>>>(W, passes, d_cyc, o);
    if (v == 2) k_chain<2><<<nb, 32>>>(W, passes, d_cyc, o);
    if (v == 3) k_chain<0, double><<<nb, 32>>>(W, passes / 4, d_cyc, o);
    if (v == 4) k_chain<2, double><<<nb, 32>>>(W, passes / 4, d_cyc, o);
    if (v == 5) k_chain_spec<<<nb, 32>>>(W, passes, d_cyc, o);
    if (v == 6) k_chain_deep3<<<nb, 32>>>(W, passes, d_cyc, o);
    if (v == 7) k_chain_pair<<<nb, 32>>>(W, passes, d_cyc, o);
    CK(cudaDeviceSynchronize());
    std::vector<long long> c(nb);
    CK(cudaMemcpy(c.data(), d_cyc, sizeof(long long) * nb, cudaMemcpyDeviceToHost));
    const int np = v == 3 || v == 4 ? passes / 4 : passes;
    std::printf("sequential WL step, %-38s %6.1f clk per trial\n", names[v], median(c) / ((double)np * kSteps));
    if (v == 0 || v == 5 || v == 6) {  // these must walk the same chain
      std::vector<long long> r(nb);
      CK(cudaMemcpy(r.data(), o, sizeof(long long) * nb, cudaMemcpyDeviceToHost));
      if (v == 0) ref = r;
      else std::printf("  (same final states as the chain-only form: %s)\n", r == ref ? "yes" : "NO");
    }
  }
  CK(cudaFree(d_out));
  CK(cudaFree(d_cyc));
  return 0;
}
