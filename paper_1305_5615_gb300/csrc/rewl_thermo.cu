// rewl_thermo.cu -- canonical thermodynamics from a density of states: for
// every temperature T (k_B = 1, beta = 1/T), with the Boltzmann weights
// w(E) = g(E) exp(-beta E) taken in log space,
//   ln Z = ln sum_E w(E)              (shifted by the largest term)
//   U    = <E>,  C = beta^2 <(E - U)^2>   (two passes: mean, then centred moment)
//   F    = -T ln Z,  S = (U - F) / T.
// One CTA per temperature (and table); block reductions over the energy bins.
// rewl_thermo_jackknife adds the resampling errors over independent runs
// (join paragraph: statistical errors by resampling): the same quantities of
// the mean ln g and of every leave-one-out mean, combined into jackknife errors.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "rewl.h"
#include "rewl_ctx.h"

namespace {

__device__ __forceinline__ double block_reduce(double v, double* sh, bool is_max) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmax(v, u) : v + u;
  }
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = sh[0];
  for (int i = 1; i < nw; ++i) r = is_max ? fmax(r, sh[i]) : r + sh[i];
  return r;
}

// One CTA per (temperature, table): table blockIdx.y of n_bins values, output
// [table][temperature][5].
__global__ void k_thermo(const double* __restrict__ lng_tables, int n_bins, int e_min, int e_step,
                         const double* __restrict__ T, double* __restrict__ out_tables) {
  __shared__ double sh[32];
  const double* lng = lng_tables + (size_t)blockIdx.y * n_bins;
  double* out = out_tables + (size_t)blockIdx.y * gridDim.x * 5;
  const double t = T[blockIdx.x];
  const double beta = 1.0 / t;
  double mx = -INFINITY;
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
    const double l = lng[b];
    if (isfinite(l)) mx = fmax(mx, l - beta * (double)(e_min + b * e_step));
  }
  mx = block_reduce(mx, sh, true);
  double z = 0.0, ze = 0.0;
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
    const double l = lng[b];
    if (isfinite(l)) {
      const double E = (double)(e_min + b * e_step);
      const double wgt = exp(l - beta * E - mx);
      z += wgt;
      ze += wgt * E;
    }
  }
  z = block_reduce(z, sh, false);
  ze = block_reduce(ze, sh, false);
  const double U = ze / z;
  double zc = 0.0;
  for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
    const double l = lng[b];
    if (isfinite(l)) {
      const double E = (double)(e_min + b * e_step);
      const double d = E - U;
      zc += exp(l - beta * E - mx) * d * d;
    }
  }
  zc = block_reduce(zc, sh, false);
  if (threadIdx.x == 0) {
    const double lnZ = mx + log(z);
    const double F = -t * lnZ;
    double* o = out + 5 * (size_t)blockIdx.x;
    o[0] = lnZ;
    o[1] = U;
    o[2] = beta * beta * (zc / z);
    o[3] = F;
    o[4] = (U - F) / t;
  }
}

// Jackknife tables: [0] the mean ln g over the R runs, [1 + i] the mean
// without run i; a bin counts only where every run is finite (else -inf).
// Sums in run order.  One thread per bin.
__global__ void k_jack_tables(const double* __restrict__ runs, int R, int n_bins, double* __restrict__ tables) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  bool fin = true;
  for (int i = 0; i < R; ++i) fin = fin && isfinite(runs[(size_t)i * n_bins + b]);
  if (!fin) {
    for (int i = 0; i <= R; ++i) tables[(size_t)i * n_bins + b] = -INFINITY;
    return;
  }
  double total = runs[b];
  for (int i = 1; i < R; ++i) total = __dadd_rn(total, runs[(size_t)i * n_bins + b]);
  tables[b] = __ddiv_rn(total, (double)R);
  for (int i = 0; i < R; ++i)
    tables[(size_t)(1 + i) * n_bins + b] = __ddiv_rn(__dsub_rn(total, runs[(size_t)i * n_bins + b]), (double)(R - 1));
}

// est = quantity of the mean table; err = sqrt((R-1)/R * sum_i (Q_(i) - Qbar)^2)
// over the leave-one-out tables.  One thread per (temperature, quantity).
__global__ void k_jack_combine(const double* __restrict__ q, int R, int n_T, double* __restrict__ est,
                               double* __restrict__ err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_T * 5) return;
  const size_t stride = (size_t)n_T * 5;
  double m = q[stride + j];
  for (int i = 1; i < R; ++i) m = __dadd_rn(m, q[(size_t)(1 + i) * stride + j]);
  m = __ddiv_rn(m, (double)R);
  double ss = 0.0;
  for (int i = 0; i < R; ++i) {
    const double d = __dsub_rn(q[(size_t)(1 + i) * stride + j], m);
    ss = __dadd_rn(ss, __dmul_rn(d, d));
  }
  est[j] = q[j];
  err[j] = sqrt(__dmul_rn(__ddiv_rn((double)(R - 1), (double)R), ss));
}

rewl_status check_temperatures(const double* temperatures, int32_t n_T) {
  for (int i = 0; i < n_T; ++i)
    if (!(temperatures[i] > 0.0) || !std::isfinite(temperatures[i])) {
      rewl_set_last_error("temperatures must be positive and finite");
      return REWL_EINVAL;
    }
  return REWL_OK;
}

}  // namespace

extern "C" rewl_status rewl_thermo_jackknife(const double* lng_runs, int32_t n_runs, int32_t n_bins, int32_t e_min,
                                             int32_t e_step, const double* temperatures, int32_t n_T, double* est,
                                             double* err) {
  if (!lng_runs || !temperatures || !est || !err || n_runs < 2 || n_bins < 1 || n_T < 1 || e_step < 1 ||
      (int64_t)n_T * 5 * (n_runs + 1) > (1ll << 31)) {
    rewl_set_last_error("rewl_thermo_jackknife: invalid argument");
    return REWL_EINVAL;
  }
  if (check_temperatures(temperatures, n_T) != REWL_OK) return REWL_EINVAL;
  bool any = false;
  for (int b = 0; b < n_bins && !any; ++b) {
    bool all = true;
    for (int i = 0; i < n_runs && all; ++i) all = std::isfinite(lng_runs[(size_t)i * n_bins + b]) != 0;
    any = all;
  }
  if (!any) {
    rewl_set_last_error("rewl_thermo_jackknife: no bin is finite in every run");
    return REWL_EINVAL;
  }
  const size_t nt = (size_t)n_runs + 1;
  double *d_runs = nullptr, *d_tab = nullptr, *d_T = nullptr, *d_q = nullptr, *d_est = nullptr, *d_err = nullptr;
  rewl_status st = REWL_OK;
  if (cudaMalloc(&d_runs, sizeof(double) * n_runs * (size_t)n_bins) != cudaSuccess ||
      cudaMalloc(&d_tab, sizeof(double) * nt * n_bins) != cudaSuccess ||
      cudaMalloc(&d_T, sizeof(double) * n_T) != cudaSuccess ||
      cudaMalloc(&d_q, sizeof(double) * nt * n_T * 5) != cudaSuccess ||
      cudaMalloc(&d_est, sizeof(double) * n_T * 5) != cudaSuccess ||
      cudaMalloc(&d_err, sizeof(double) * n_T * 5) != cudaSuccess) {
    rewl_set_last_error("rewl_thermo_jackknife: device allocation failed");
    st = REWL_ENOMEM;
  }
  if (st == REWL_OK &&
      (cudaMemcpy(d_runs, lng_runs, sizeof(double) * n_runs * (size_t)n_bins, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_T, temperatures, sizeof(double) * n_T, cudaMemcpyHostToDevice) != cudaSuccess)) {
    rewl_set_last_error("rewl_thermo_jackknife: copy failed");
    st = REWL_ECUDA;
  }
  if (st == REWL_OK) {
    k_jack_tables<<<(n_bins + 255) / 256, 256>>>(d_runs, n_runs, n_bins, d_tab);
    k_thermo<<<dim3(n_T, (unsigned)nt), 256>>>(d_tab, n_bins, e_min, e_step, d_T, d_q);
    k_jack_combine<<<(n_T * 5 + 127) / 128, 128>>>(d_q, n_runs, n_T, d_est, d_err);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(est, d_est, sizeof(double) * n_T * 5, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(err, d_err, sizeof(double) * n_T * 5, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rewl_set_last_error("rewl_thermo_jackknife: kernel failed");
      st = REWL_ECUDA;
    }
  }
  cudaFree(d_runs);
  cudaFree(d_tab);
  cudaFree(d_T);
  cudaFree(d_q);
  cudaFree(d_est);
  cudaFree(d_err);
  return st;
}

extern "C" rewl_status rewl_thermo(const double* lng, int32_t n_bins, int32_t e_min, int32_t e_step,
                                   const double* temperatures, int32_t n_T, double* out) {
  if (!lng || !temperatures || !out || n_bins < 1 || n_T < 1 || e_step < 1) {
    rewl_set_last_error("rewl_thermo: invalid argument");
    return REWL_EINVAL;
  }
  if (check_temperatures(temperatures, n_T) != REWL_OK) return REWL_EINVAL;
  bool any = false;
  for (int b = 0; b < n_bins; ++b) any |= std::isfinite(lng[b]) != 0;
  if (!any) {
    rewl_set_last_error("rewl_thermo: no finite ln g");
    return REWL_EINVAL;
  }
  double *d_lng = nullptr, *d_T = nullptr, *d_out = nullptr;
  rewl_status st = REWL_OK;
  if (cudaMalloc(&d_lng, sizeof(double) * n_bins) != cudaSuccess || cudaMalloc(&d_T, sizeof(double) * n_T) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(double) * 5 * n_T) != cudaSuccess) {
    rewl_set_last_error("rewl_thermo: device allocation failed");
    st = REWL_ENOMEM;
  }
  if (st == REWL_OK && (cudaMemcpy(d_lng, lng, sizeof(double) * n_bins, cudaMemcpyHostToDevice) != cudaSuccess ||
                        cudaMemcpy(d_T, temperatures, sizeof(double) * n_T, cudaMemcpyHostToDevice) != cudaSuccess)) {
    rewl_set_last_error("rewl_thermo: copy failed");
    st = REWL_ECUDA;
  }
  if (st == REWL_OK) {
    k_thermo<<<dim3(n_T, 1), 256>>>(d_lng, n_bins, e_min, e_step, d_T, d_out);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d_out, sizeof(double) * 5 * n_T, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rewl_set_last_error("rewl_thermo: kernel failed");
      st = REWL_ECUDA;
    }
  }
  cudaFree(d_lng);
  cudaFree(d_T);
  cudaFree(d_out);
  return st;
}
