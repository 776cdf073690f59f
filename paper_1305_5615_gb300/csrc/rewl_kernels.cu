// rewl_kernels.cu -- the device phases of replica-exchange Wang-Landau:
//   k_init_lattice  random start configurations and their energies
//   k_descent       +-J: zero-temperature descent that fixes the energy range
//   k_entry         greedy walk of every walker into its window
//   k_sweep         the WL walk (paper, WL paragraph) -- the hot loop
//   k_exchange      configuration swaps between neighbouring windows, Eq. (1)
//   k_flat_merge    per-walker flatness, averaging of the window's ln g,
//                   f -> sqrt f and termination (paragraph after Eq. (1))
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>

#include "rewl_device.cuh"
#include "rewl_kernels.h"
#include "rewl_layout.h"

namespace rewl {

// ---------------------------------------------------------------------------
// Generic single-site helpers on a walker's packed configuration in global
// memory (used by the one-off set-up kernels).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t g_site(const Problem& P, const uint32_t* lat, int x, int y) {
  if (P.model == kPotts) return (lat[y * P.Wr + (x >> 3)] >> ((x & 7) * 4)) & 15u;
  return (lat[y * P.Wr + (x >> 5)] >> (x & 31)) & 1u;
}
__device__ __forceinline__ void g_set_site(const Problem& P, uint32_t* lat, int x, int y, uint32_t v) {
  if (P.model == kPotts) {
    uint32_t& wd = lat[y * P.Wr + (x >> 3)];
    const int sh = (x & 7) * 4;
    wd = (wd & ~(15u << sh)) | (v << sh);
  } else {
    uint32_t& wd = lat[y * P.Wr + (x >> 5)];
    wd = (wd & ~(1u << (x & 31))) | (v << (x & 31));
  }
}
// bond energy: Ising / +-J -J s_a s_b (bit 1 = spin -1, coupling bit 1 = J -1); Potts -delta
__device__ __forceinline__ int bond_e(const Problem& P, uint32_t a, uint32_t b, uint32_t jneg) {
  if (P.model == kPotts) return a == b ? -1 : 0;
  return ((a ^ b ^ jneg) & 1u) ? 1 : -1;
}
// coupling bit of plane (0 right, 1 down, 2 behind) at (x, row); row = y in 2D, z L + y in 3D
__device__ __forceinline__ uint32_t g_jbit(const Problem& P, const uint32_t* J, int plane, int x, int row) {
  if (P.model != kEA && P.model != kEA3) return 0u;
  return coupling_bit(J, P.Wr1, plane, P.rows, x, row);
}
__device__ int g_energy(const Problem& P, const uint32_t* lat, const uint32_t* J) {
  int E = 0;
  const int L = P.L, nz = P.model == kEA3 ? L : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < L; ++y)
      for (int x = 0; x < L; ++x) {
        const int row = z * L + y;
        const uint32_t s = g_site(P, lat, x, row);
        const int xr = x + 1 == L ? 0 : x + 1, yd = y + 1 == L ? 0 : y + 1;
        E += bond_e(P, s, g_site(P, lat, xr, row), g_jbit(P, J, 0, x, row));
        E += bond_e(P, s, g_site(P, lat, x, z * L + yd), g_jbit(P, J, 1, x, row));
        if (P.model == kEA3) {
          const int zb = z + 1 == L ? 0 : z + 1;
          E += bond_e(P, s, g_site(P, lat, x, zb * L + y), g_jbit(P, J, 2, x, row));
        }
      }
  return E;
}
// energy change when site (x, y, z) takes value v (z = 0 in 2D)
__device__ int g_delta_e(const Problem& P, const uint32_t* lat, const uint32_t* J, int x, int y, int z, uint32_t v) {
  const int L = P.L;
  const int xl = x ? x - 1 : L - 1, xr = x + 1 == L ? 0 : x + 1;
  const int yu = y ? y - 1 : L - 1, yd = y + 1 == L ? 0 : y + 1;
  const int zo = z * L, row = zo + y;
  const uint32_t s = g_site(P, lat, x, row);
  const uint32_t nr = g_site(P, lat, xr, row), nl = g_site(P, lat, xl, row);
  const uint32_t nd = g_site(P, lat, x, zo + yd), nu = g_site(P, lat, x, zo + yu);
  const uint32_t jr = g_jbit(P, J, 0, x, row), jl = g_jbit(P, J, 0, xl, row);
  const uint32_t jd = g_jbit(P, J, 1, x, row), ju = g_jbit(P, J, 1, x, zo + yu);
  int before = bond_e(P, s, nr, jr) + bond_e(P, s, nl, jl) + bond_e(P, s, nd, jd) + bond_e(P, s, nu, ju);
  int after = bond_e(P, v, nr, jr) + bond_e(P, v, nl, jl) + bond_e(P, v, nd, jd) + bond_e(P, v, nu, ju);
  if (P.model == kEA3) {
    const int zf = z ? z - 1 : L - 1, zb = z + 1 == L ? 0 : z + 1;
    const uint32_t nb = g_site(P, lat, x, zb * L + y), nf = g_site(P, lat, x, zf * L + y);
    const uint32_t jb = g_jbit(P, J, 2, x, row), jf = g_jbit(P, J, 2, x, zf * L + y);
    before += bond_e(P, s, nb, jb) + bond_e(P, s, nf, jf);
    after += bond_e(P, v, nb, jb) + bond_e(P, v, nf, jf);
  }
  return after - before;
}

// The site of a draw: (x, y) on the square lattice, (x, y, z) on the cube.
__device__ __forceinline__ void decode_site(const Problem& P, uint32_t site, int& x, int& y, int& z) {
  if (P.model == kEA3) {
    z = (int)mulhi32(site, P.magic_L2);
    site -= (uint32_t)z * (uint32_t)(P.L * P.L);
  } else {
    z = 0;
  }
  y = (int)mulhi32(site, P.magic_L);
  x = (int)site - y * P.L;
}

__device__ __forceinline__ void propose(const Problem& P, const uint32_t* lat, const U4& r, int& x, int& y, int& z,
                                        uint32_t& v) {
  const uint32_t site = scale32(r.x, (uint32_t)P.N);
  decode_site(P, site, x, y, z);
  const uint32_t s = g_site(P, lat, x, z * P.L + y);
  if (P.model == kPotts) {
    v = s + 1u + scale32(r.y, (uint32_t)(P.q - 1));
    if (v >= (uint32_t)P.q) v -= (uint32_t)P.q;
  } else {
    v = s ^ 1u;
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels (one thread per walker)
// ---------------------------------------------------------------------------
__global__ void k_init_lattice(Problem P, DevState S) {
  const int W = blockIdx.x * blockDim.x + threadIdx.x;
  if (W >= P.n_walkers) return;
  uint32_t* lat = S.lat + (size_t)W * P.lat_words;
  for (int i = 0; i < P.lat_words; ++i) lat[i] = 0u;
  U4 r{0, 0, 0, 0};
  for (int i = 0; i < P.N; ++i) {
    const int x = i % P.L, y = i / P.L;
    if (P.model == kPotts) {
      if ((i & 3) == 0) r = philox10((uint32_t)(i >> 2), 0u, (uint32_t)W, kTagInit, P.seed_lo, P.seed_hi);
      const uint32_t w = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
      g_set_site(P, lat, x, y, scale32(w, (uint32_t)P.q));
    } else {
      if ((i & 127) == 0) r = philox10((uint32_t)(i >> 7), 0u, (uint32_t)W, kTagInit, P.seed_lo, P.seed_hi);
      const int wi = (i & 127) >> 5;
      const uint32_t w = wi == 0 ? r.x : wi == 1 ? r.y : wi == 2 ? r.z : r.w;
      g_set_site(P, lat, x, y, (w >> (i & 31)) & 1u);
    }
  }
  S.E[W] = g_energy(P, lat, S.J);
  S.entry_t[W] = 0;
  S.status[W] = 0;
}

__device__ __forceinline__ int window_distance(int E, int lo, int hi) { return E < lo ? lo - E : (E > hi ? E - hi : 0); }

// Bins of window a: its own width (run-time balanced windows of unequal width,
// Fig. 1b), or P.w for every window when no table is given (Fig. 1a).  P.w is
// always the largest width and the stride of the per-walker ln g and H rows.
__device__ __forceinline__ int window_width(const Problem& P, const DevState& S, int a) {
  return S.win_width ? S.win_width[a] : P.w;
}

// One greedy move on the entry stream.  target < 0: minimise E (descent);
// otherwise minimise the distance to window `target`.
__device__ void greedy_move(const Problem& P, DevState& S, uint32_t* lat, int W, int lo, int hi, bool descent) {
  const uint64_t t = S.entry_t[W]++;
  const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagEntry, P.seed_lo, P.seed_hi);
  int x, y, z;
  uint32_t v;
  propose(P, lat, r, x, y, z, v);
  const int E = S.E[W];
  const int En = E + g_delta_e(P, lat, S.J, x, y, z, v);
  const int before = descent ? E : window_distance(E, lo, hi);
  const int after = descent ? En : window_distance(En, lo, hi);
  if (after <= before) {
    g_set_site(P, lat, x, z * P.L + y, v);
    S.E[W] = En;
  }
}

__global__ void k_descent(Problem P, DevState S, uint64_t n_att) {
  const int W = blockIdx.x * blockDim.x + threadIdx.x;
  if (W >= P.n_walkers) return;
  uint32_t* lat = S.lat + (size_t)W * P.lat_words;
  for (uint64_t n = 0; n < n_att; ++n) greedy_move(P, S, lat, W, 0, 0, true);
}

__global__ void k_entry(Problem P, DevState S, uint64_t budget) {
  const int W = blockIdx.x * blockDim.x + threadIdx.x;
  if (W >= P.n_walkers) return;
  uint32_t* lat = S.lat + (size_t)W * P.lat_words;
  const int a = W / P.m;
  const int lo = P.e_min + S.win_start[a] * P.e_step;
  const int hi = P.e_min + (S.win_start[a] + window_width(P, S, a) - 1) * P.e_step;
  for (uint64_t n = 0; n < budget && window_distance(S.E[W], lo, hi) > 0; ++n) greedy_move(P, S, lat, W, lo, hi, false);
  if (window_distance(S.E[W], lo, hi) == 0) return;
  for (int i = 0; i < P.lat_words; ++i) lat[i] = S.seed_config[i];
  S.E[W] = g_energy(P, lat, S.J);
  for (uint64_t n = 0; n < budget && window_distance(S.E[W], lo, hi) > 0; ++n) greedy_move(P, S, lat, W, lo, hi, false);
  if (window_distance(S.E[W], lo, hi) != 0) S.status[W] = 5;  // REWL_EENTRY
}

// ---------------------------------------------------------------------------
// The WL sweep kernel.
//
// G lanes run one walker.  For every group of G consecutive trials each lane
// draws one trial (Philox, site, proposed Potts value, float log of u) in
// parallel; the G trials are then applied in order, every lane of the group
// executing the same (redundant) sequential step.  The walker's
// configuration, the fixed-point shadow of its ln g (units of 2^-40) and its
// H live in shared memory, interleaved by walker.  The acceptance test
//      accept iff ln g(E_old) - ln g(E_new) >= ln u         (min[1, g_old/g_new])
// is decided on the shadow against float ln u whenever the two differ by more
// than the guard band; otherwise (rarely) it is recomputed exactly in FP64
// from the stored doubles, as the plain definition does.  The FP64 ln g is
// brought up to date at the end of the launch by exact integer emulation of
// the per-visit additions ln g += ln f (add_pow2_repeated), so the hot loop
// issues no FP64 instruction.
// ---------------------------------------------------------------------------
// Site and proposal of a trial from its draw: (x, y) and the Potts offset on
// the square lattice; (x, y) and z (carried in pv) on the cube.
template <int MODEL>
__device__ __forceinline__ void trial_site(const Problem& P, const U4& r, int& x, int& y, uint32_t& pv) {
  const uint32_t site = scale32(r.x, (uint32_t)P.N);
  if constexpr (MODEL == kEA3) {
    const uint32_t z = mulhi32(site, P.magic_L2);
    const uint32_t rem = site - z * (uint32_t)(P.L * P.L);
    y = (int)mulhi32(rem, P.magic_L);
    x = (int)rem - y * P.L;
    pv = z;
  } else {
    y = (int)mulhi32(site, P.magic_L);
    x = (int)site - y * P.L;
    pv = MODEL == kPotts ? scale32(r.y, (uint32_t)(P.q - 1)) : 0u;
  }
}

// Bit k set iff trial k < lane of this group of G moves a site of this
// trial's neighbourhood (the site and its 4, or on the cube 6, neighbours).
template <int MODEL, int G>
__device__ __forceinline__ uint32_t conflict_mask(const Problem& P, int x, int y, uint32_t pv, int lane,
                                                  uint32_t gm) {
  const int L = P.L;
  const int xl = x ? x - 1 : L - 1, xr = x + 1 == L ? 0 : x + 1;
  const int yu = y ? y - 1 : L - 1, yd = y + 1 == L ? 0 : y + 1;
  const uint32_t zk = MODEL == kEA3 ? pv << 16 : 0u;
  const uint32_t key = (uint32_t)x | ((uint32_t)y << 8) | zk;
  const uint32_t kl = (uint32_t)xl | ((uint32_t)y << 8) | zk, kr = (uint32_t)xr | ((uint32_t)y << 8) | zk;
  const uint32_t ku = (uint32_t)x | ((uint32_t)yu << 8) | zk, kd = (uint32_t)x | ((uint32_t)yd << 8) | zk;
  uint32_t kf = key, kb = key;
  if constexpr (MODEL == kEA3) {
    const uint32_t z = pv, zf = z ? z - 1 : (uint32_t)L - 1, zb = z + 1 == (uint32_t)L ? 0u : z + 1;
    kf = (uint32_t)x | ((uint32_t)y << 8) | (zf << 16);
    kb = (uint32_t)x | ((uint32_t)y << 8) | (zb << 16);
  }
  uint32_t M = 0;
#pragma unroll
  for (int i = 0; i < G - 1; ++i) {
    const uint32_t pi = __shfl_sync(gm, key, i, G);
    bool hit = pi == key || pi == kl || pi == kr || pi == ku || pi == kd;
    if constexpr (MODEL == kEA3) hit = hit || pi == kf || pi == kb;
    M |= (hit && i < lane) ? (1u << i) : 0u;
  }
  return M;
}

template <int G>
__device__ __forceinline__ uint32_t group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    const uint32_t lane = threadIdx.x & 31u;
    return ((1u << G) - 1u) << (lane & ~(uint32_t)(G - 1));
  }
}

template <int G, typename T>
__device__ __forceinline__ T gshfl(uint32_t mask, T v, int src) {
  if constexpr (G == 1) {
    return v;
  } else if constexpr (sizeof(T) == 8) {
    const long long b = __shfl_sync(mask, (long long)v, src, G);
    return (T)b;
  } else {
    return __shfl_sync(mask, v, src, G);
  }
}

template <int G>
__device__ __forceinline__ void gsync(uint32_t mask) {
  if constexpr (G > 1) __syncwarp(mask);
}

// exact FP64 re-evaluation of one acceptance test (rare)
__device__ __noinline__ bool exact_accept(const DevState& S, const Problem& P, int W, int k, int bin, uint32_t h_cur,
                                          int bn, uint32_t h_new, uint64_t k52, uint64_t& n_tie) {
  const double* lngW = S.lng + (size_t)W * P.w;
  const uint32_t* HW = S.H + (size_t)W * P.w;
  const uint64_t vc = add_pow2_repeated(double_to_bits(lngW[bin]), k, h_cur - HW[bin]);
  const uint64_t vn = add_pow2_repeated(double_to_bits(lngW[bn]), k, h_new - HW[bn]);
  const double delta = __dsub_rn(bits_to_double(vc), bits_to_double(vn));
  if (delta >= 0.0) return true;
  const double u = __dmul_rn(__ull2double_rn(2ull * k52 + 1ull), 0x1p-53);
  const double lu = log(u);
  if (fabs(__dsub_rn(lu, delta)) < 1e-12) ++n_tie;
  return lu < delta;
}

// ---------------------------------------------------------------------------
// The WL sweep kernel, speculative form (G = 8, 16 or 32 lanes per walker).
//
// Same trials, same order, same results as k_sweep; only the work is split
// differently.  For a group of G consecutive trials every lane evaluates its
// own trial against the configuration as it stands when the group starts:
// the Philox draw, the site, the proposed value, the energy change (as a bin
// offset) and ln u.  It also records which earlier trials of the group touch
// its site or a neighbour (mask M_j).  The trials are then applied in order;
// a trial whose mask meets an earlier *accepted* trial is re-evaluated on the
// current configuration, all others use the speculative offset.  What stays
// sequential is the chain bin -> ln g shadow of the new bin -> acceptance.
// ---------------------------------------------------------------------------
template <int MODEL>
struct TrialEval {
  int dbin;          // (E_new - E_old) / e_step
  uint32_t widx;     // lattice word (shared-memory index) the move writes
  uint32_t wmask;    // Ising / +-J: bit to flip;  Potts: nibble shift (low 8 bits) | new value << 8
  uint32_t delta;    // the move as an XOR on the word: Ising / +-J the bit; Potts (old ^ new value) << shift
};

template <int MODEL>
__device__ __forceinline__ TrialEval<MODEL> eval_trial(const Problem& P, const uint32_t* s_lat, const uint32_t* s_J,
                                                       int wpb, int lw, int x, int y, uint32_t pv) {
  const int L = P.L, Wr = P.Wr;
  const int xl = x ? x - 1 : L - 1, xr = x + 1 == L ? 0 : x + 1;
  const int yu = y ? y - 1 : L - 1, yd = y + 1 == L ? 0 : y + 1;
  TrialEval<MODEL> t;
  if constexpr (MODEL == kEA3) {  // the cube: pv carries z, rows are z * L + y
    const int z = (int)pv, zo = z * L, row = zo + y;
    const int zf = z ? z - 1 : L - 1, zb = z + 1 == L ? 0 : z + 1;
    const uint32_t c = spin_bit(s_lat, wpb, lw, Wr, x, row);
    const uint32_t nr = spin_bit(s_lat, wpb, lw, Wr, xr, row), nl = spin_bit(s_lat, wpb, lw, Wr, xl, row);
    const uint32_t nd = spin_bit(s_lat, wpb, lw, Wr, x, zo + yd), nu = spin_bit(s_lat, wpb, lw, Wr, x, zo + yu);
    const uint32_t nb = spin_bit(s_lat, wpb, lw, Wr, x, zb * L + y), nf = spin_bit(s_lat, wpb, lw, Wr, x, zf * L + y);
    const int R = P.rows;
    const uint32_t jr = coupling_bit(s_J, P.Wr1, 0, R, x, row), jl = coupling_bit(s_J, P.Wr1, 0, R, xl, row);
    const uint32_t jd = coupling_bit(s_J, P.Wr1, 1, R, x, row), ju = coupling_bit(s_J, P.Wr1, 1, R, x, zo + yu);
    const uint32_t jb = coupling_bit(s_J, P.Wr1, 2, R, x, row), jf = coupling_bit(s_J, P.Wr1, 2, R, x, zf * L + y);
    const int sat = (int)(((c ^ nr ^ jr) & 1u) == 0) + (int)(((c ^ nl ^ jl) & 1u) == 0) +
                    (int)(((c ^ nd ^ jd) & 1u) == 0) + (int)(((c ^ nu ^ ju) & 1u) == 0) +
                    (int)(((c ^ nb ^ jb) & 1u) == 0) + (int)(((c ^ nf ^ jf) & 1u) == 0);
    t.dbin = sat - 3;  // dE = 4 * satisfied - 12
    t.widx = (uint32_t)((row * Wr + (x >> 5)) * wpb + lw);
    t.wmask = 1u << (x & 31);
    t.delta = t.wmask;
  } else if constexpr (MODEL == kPotts) {
    const uint32_t v = potts_val(s_lat, wpb, lw, Wr, x, y);
    uint32_t nv = v + 1u + pv;
    if (nv >= (uint32_t)P.q) nv -= (uint32_t)P.q;
    const uint32_t n1 = potts_val(s_lat, wpb, lw, Wr, xr, y), n2 = potts_val(s_lat, wpb, lw, Wr, xl, y);
    const uint32_t n3 = potts_val(s_lat, wpb, lw, Wr, x, yd), n4 = potts_val(s_lat, wpb, lw, Wr, x, yu);
    t.dbin = (int)(n1 == v) + (int)(n2 == v) + (int)(n3 == v) + (int)(n4 == v) - (int)(n1 == nv) - (int)(n2 == nv) -
             (int)(n3 == nv) - (int)(n4 == nv);
    t.widx = (uint32_t)((y * Wr + (x >> 3)) * wpb + lw);
    t.wmask = (uint32_t)((x & 7) * 4) | (nv << 8);
    t.delta = (v ^ nv) << ((x & 7) * 4);
  } else {
    const uint32_t c = spin_bit(s_lat, wpb, lw, Wr, x, y);
    const uint32_t nr = spin_bit(s_lat, wpb, lw, Wr, xr, y), nl = spin_bit(s_lat, wpb, lw, Wr, xl, y);
    const uint32_t nd = spin_bit(s_lat, wpb, lw, Wr, x, yd), nu = spin_bit(s_lat, wpb, lw, Wr, x, yu);
    uint32_t jr = 0, jl = 0, jd = 0, ju = 0;
    if constexpr (MODEL == kEA) {
      jr = coupling_bit(s_J, P.Wr1, 0, L, x, y);
      jl = coupling_bit(s_J, P.Wr1, 0, L, xl, y);
      jd = coupling_bit(s_J, P.Wr1, 1, L, x, y);
      ju = coupling_bit(s_J, P.Wr1, 1, L, x, yu);
    }
    const int sat = (int)(((c ^ nr ^ jr) & 1u) == 0) + (int)(((c ^ nl ^ jl) & 1u) == 0) +
                    (int)(((c ^ nd ^ jd) & 1u) == 0) + (int)(((c ^ nu ^ ju) & 1u) == 0);
    t.dbin = sat - 2;  // dE = 4 * satisfied - 8
    t.widx = (uint32_t)((y * Wr + (x >> 5)) * wpb + lw);
    t.wmask = 1u << (x & 31);
    t.delta = t.wmask;
  }
  return t;
}

// One staged trial: what the parallel phase hands to the sequential phase.
struct StagedTrial {
  uint32_t pk;     // dbin + 8 | pv << 8 | x << 16 | y << 24
  uint32_t mask;   // earlier trials of the group whose site lies in this trial's 5-site neighbourhood
  uint32_t widx;   // lattice word the move writes (shared-memory index)
  uint32_t wmask;  // Ising / +-J: bit to flip;  Potts: nibble shift | new value << 8
  int64_t thr;     // ln u in units of 2^-40 (float log; see kGuardFx)
};

// The chain forms split a staged trial in two: what the sequential step reads
// for every trial (16 bytes, one shared-memory load) and the move itself, which
// the sequential step does not touch: accepted moves are written to the
// configuration by their own lanes after the group (an XOR per move), except
// where a later trial of the group needs the configuration they leave.  Both
// arrays are laid out [trial of the group][walker of the CTA], so that the
// walkers of one warp (lane 0 of each group of G lanes) read their trial j
// from neighbouring addresses.
struct __align__(16) HotTrial {
  int64_t thr;     // ln u - j ln f in units of 2^-40 (j: the trial's index in its group; see below)
  int16_t dbin;    // (E_new - E_old) / e_step on the configuration the group started from
  uint16_t j;      // the trial's index in its group
  uint32_t mask;   // earlier trials of the group whose site lies in this trial's neighbourhood
};
struct ColdTrial {
  uint32_t widx;   // lattice word the move writes
  uint32_t delta;  // the move as an XOR on that word
  uint32_t site;   // x | y << 8 | pv << 16 (for the re-evaluation of a conflicting trial)
};
static_assert(sizeof(HotTrial) == 16 && sizeof(ColdTrial) == 12, "staging size");
constexpr size_t kChainStagingBytes = sizeof(HotTrial) + sizeof(ColdTrial);  // per walker and trial of a group

template <int MODEL, int G>
__global__ void __launch_bounds__(256) k_sweep_spec(Problem P, DevState S, SweepLaunch A) {
  static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32, "G");
  extern __shared__ __align__(16) unsigned char smem[];
  const int wpb = A.wpb;
  StagedTrial* s_stage = reinterpret_cast<StagedTrial*>(smem);                 // [wpb][G]
  int64_t* s_fx = reinterpret_cast<int64_t*>(s_stage + (G > 1 ? (size_t)wpb * G : 0));
  uint32_t* s_H = reinterpret_cast<uint32_t*>(s_fx + (size_t)P.w * wpb);
  uint32_t* s_lat = s_H + (size_t)P.w * wpb;
  uint32_t* s_J = s_lat + (size_t)P.lat_words * wpb;
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const int first = blockIdx.x * wpb;
  const int nloc = min(wpb, A.n_active - first);

  for (int i = tid; i < nloc * P.w; i += nthr) {
    const int l = i / P.w, b = i - l * P.w;
    const size_t g = (size_t)S.active[first + l] * P.w + b;
    s_fx[b * wpb + l] = to_fx(double_to_bits(S.lng[g]));
    s_H[b * wpb + l] = S.H[g];
  }
  for (int i = tid; i < nloc * P.lat_words; i += nthr) {
    const int l = i / P.lat_words, j = i - l * P.lat_words;
    s_lat[j * wpb + l] = S.lat[(size_t)S.active[first + l] * P.lat_words + j];
  }
  if (MODEL == kEA || MODEL == kEA3)
    for (int i = tid; i < P.j_words; i += nthr) s_J[i] = S.J[i];
  __syncthreads();

  const int lw = tid / G, lane = tid % G;
  bool valid = lw < nloc;
  int W = 0, a = 0, bin = 0, kexp = 0, wstart = 0;
  if (valid) {
    W = S.active[first + lw];
    a = W / P.m;
    wstart = S.win_start[a];
    bin = (S.E[W] - P.e_min) / P.e_step - wstart;
    kexp = lnf_exponent(S.lnf[a]);
    if ((unsigned)bin >= (unsigned)window_width(P, S, a) || kexp == kBadLnf) {
      if (lane == 0) S.status[W] = kWalkerBadInput;
      valid = false;
    }
  }
  if (valid) {
    const int64_t lnf_fx = 1ll << (kFxBits - kexp);
    int64_t fx_cur = s_fx[bin * wpb + lw];
    uint32_t h_cur = s_H[bin * wpb + lw];
    uint64_t n_acc = 0, n_tie = 0, n_exact = 0;
    const uint32_t gm = group_mask<G>();
    const int w = window_width(P, S, a);  // the window test; P.w is the layout stride
    const uint64_t t0 = S.clock[0] * (uint64_t)P.N;
    StagedTrial* my_stage = s_stage + (size_t)lw * G;

    for (uint32_t base = 0; base < A.n_att; base += G) {
      // ---- parallel phase: lane l evaluates trial base + l on the current configuration
      StagedTrial tr;
      {
        const uint64_t t = t0 + base + (uint32_t)lane;
        const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
        int x, y;
        uint32_t pv;
        trial_site<MODEL>(P, r, x, y, pv);
        const float uf = __ull2float_rn(2ull * u52_bits(r.z, r.w) + 1ull) * 0x1p-53f;
        tr.thr = __float2ll_rn(logf(uf) * 1099511627776.0f);
        const TrialEval<MODEL> ev = eval_trial<MODEL>(P, s_lat, s_J, wpb, lw, x, y, pv);
        const uint32_t pk = (uint32_t)x | ((uint32_t)y << 8);
        uint32_t M = 0;
        if constexpr (G > 1) M = conflict_mask<MODEL, G>(P, x, y, pv, lane, gm);
        tr.pk = (uint32_t)(ev.dbin + 8) | (pv << 8) | (pk << 16);
        tr.mask = M;
        tr.widx = ev.widx;
        tr.wmask = ev.wmask;
        if constexpr (G > 1) my_stage[lane] = tr;
      }
      if constexpr (G > 1) __syncwarp(gm);  // staged trials visible to lane 0

      // ---- sequential phase: lane 0 applies the trials in order
      if (lane == 0) {
        const int n_here = (int)min((uint32_t)G, A.n_att - base);
        uint32_t accm = 0;
        StagedTrial nxt = tr;
        if constexpr (G > 1) nxt = my_stage[0];
#pragma unroll 1
        for (int j = 0; j < n_here; ++j) {
          const StagedTrial cur = nxt;
          if constexpr (G > 1) {
            if (j + 1 < n_here) nxt = my_stage[j + 1];  // prefetch the next staged trial
          }
          int dbin = (int)(cur.pk & 0xffu) - 8;
          uint32_t widx = cur.widx, wmask = cur.wmask;
          if constexpr (G > 1) {
            if (accm & cur.mask) {  // an accepted earlier trial touched this neighbourhood: re-evaluate
              const TrialEval<MODEL> e2 = eval_trial<MODEL>(P, s_lat, s_J, wpb, lw, (int)((cur.pk >> 16) & 0xffu),
                                                           (int)(cur.pk >> 24), (cur.pk >> 8) & 0xffu);
              dbin = e2.dbin;
              widx = e2.widx;
              wmask = e2.wmask;
            }
          }
          const int bn = bin + dbin;
          const bool inwin = (unsigned)bn < (unsigned)w;
          const int bl = inwin ? bn : bin;
          const int64_t fxn = s_fx[bl * wpb + lw];
          const uint32_t hn = s_H[bl * wpb + lw];
          const int64_t d = (fx_cur - fxn) - cur.thr;
          bool acc = dbin == 0 || (inwin && d > kGuardFx);
          if (dbin != 0 && inwin && d >= -kGuardFx && d <= kGuardFx) {  // rare: exact FP64 test
            const uint64_t t = t0 + base + (uint32_t)j;
            const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
            acc = exact_accept(S, P, W, kexp, bin, h_cur, bn, hn, u52_bits(r.z, r.w), n_tie);
            ++n_exact;
          }
          // branch-free update: configuration word, write-back of the bin left, new state
          const bool mv = acc && dbin != 0;
          const uint32_t word = s_lat[widx];
          uint32_t nword;
          if constexpr (MODEL == kPotts) {
            const uint32_t sh = wmask & 0xffu, nv = wmask >> 8;
            nword = (word & ~(15u << sh)) | (nv << sh);
          } else {
            nword = word ^ wmask;
          }
          s_lat[widx] = acc ? nword : word;
          const int wb = (mv ? bin : bl) * wpb + lw;  // write-back target (a harmless rewrite of bl when no move)
          s_fx[wb] = mv ? fx_cur : fxn;
          s_H[wb] = mv ? h_cur : hn;
          accm |= (uint32_t)acc << j;
          n_acc += acc;
          bin = mv ? bn : bin;
          fx_cur = mv ? fxn : fx_cur;
          h_cur = mv ? hn : h_cur;
          fx_cur += lnf_fx;  // ln g(E) += ln f on the shadow
          ++h_cur;           // H(E) += 1
        }
      }
      if constexpr (G > 1) __syncwarp(gm);  // lane 0's configuration updates visible to the group
    }
    if (lane == 0) {
      s_fx[bin * wpb + lw] = fx_cur;
      s_H[bin * wpb + lw] = h_cur;
      S.E[W] = P.e_min + (wstart + bin) * P.e_step;
      S.wl_accept[W] += n_acc;
      S.near_ties[W] += n_tie;
      S.exact_tests[W] += n_exact;
    }
  }
  __syncthreads();

  for (int i = tid; i < nloc * P.w; i += nthr) {
    const int l = i / P.w, b = i - l * P.w;
    const int Wl = S.active[first + l];
    const size_t g = (size_t)Wl * P.w + b;
    const uint32_t hs = s_H[b * wpb + l];
    const uint32_t c = hs - S.H[g];
    const int kx = lnf_exponent(S.lnf[Wl / P.m]);
    if (c && kx != kBadLnf) {
      S.lng[g] = bits_to_double(add_pow2_repeated(double_to_bits(S.lng[g]), kx, c));
      S.H[g] = hs;
    }
  }
  for (int i = tid; i < nloc * P.lat_words; i += nthr) {
    const int l = i / P.lat_words, j = i - l * P.lat_words;
    S.lat[(size_t)S.active[first + l] * P.lat_words + j] = s_lat[j * wpb + l];
  }
}

// ---------------------------------------------------------------------------
// The WL sweep kernel, two-deep chain form.  Same trials, order and results
// as k_sweep_spec; the sequential phase is reorganised around its critical
// path.  While trial j resolves, lane 0 already loads the ln g shadow of both
// bins trial j+1 can target (from the current bin, and from trial j's new
// bin); once trial j's outcome is known one of the two is selected, with the
// register value forwarded when the target is the bin trial j just left.
// The sequential step does not write the configuration: after each group the
// lanes write their own accepted moves (one XOR each), and a trial that meets
// an earlier accepted one first writes the moves its neighbourhood depends on.
// H is not kept during the launch: the shadow of a bin grows by exactly
// ln f (in 2^-40 units) per visit, so the visit count of every bin is
// (shadow_end - shadow_start) / ln f, and the write-back adds it to H and
// applies the same number of FP64 additions to ln g.  The shadow array
// carries kGuardBins unused bins on each side so that speculative loads
// need no clamping: the current bin is always inside the window, one
// trial moves at most 4 bins (Potts; 3 on the cube, 2 for Ising and the 2D
// glass), and the furthest load, trial j+1's target after a move of trial
// j, is two such offsets away.
// ---------------------------------------------------------------------------
constexpr int kGuardBins = 8;

// exact FP64 re-evaluation from visit counts reconstructed from the shadow
__device__ __noinline__ bool exact_accept_fx(const DevState& S, const Problem& P, int W, int k, int bin,
                                             int64_t fx_cur, int bn, int64_t fx_new, uint64_t k52, uint64_t& n_tie) {
  const double* lngW = S.lng + (size_t)W * P.w;
  const int sh = kFxBits - k;
  const uint64_t vc0 = double_to_bits(lngW[bin]), vn0 = double_to_bits(lngW[bn]);
  const uint32_t cc = (uint32_t)((fx_cur - to_fx(vc0)) >> sh);
  const uint32_t cn = (uint32_t)((fx_new - to_fx(vn0)) >> sh);
  const double vc = bits_to_double(add_pow2_repeated(vc0, k, cc));
  const double vn = bits_to_double(add_pow2_repeated(vn0, k, cn));
  const double delta = __dsub_rn(vc, vn);
  if (delta >= 0.0) return true;
  const double u = __dmul_rn(__ull2double_rn(2ull * k52 + 1ull), 0x1p-53);
  const double lu = log(u);
  if (fabs(__dsub_rn(lu, delta)) < 1e-12) ++n_tie;
  return lu < delta;
}

// ---------------------------------------------------------------------------
// Warp-specialised form (variant kSweepRing): a producer warp computes the
// draws of upcoming groups (Philox, site, Potts offset, ln u, conflict mask)
// into a ring of kRingSlots groups in shared memory while the walker's warp
// runs the sequential chain; the walker's warp only evaluates the moves on the
// current configuration.  The two warps sit on different SM sub-partitions,
// so the producer does not take issue slots from the chain.  Hand-off through
// mbarriers: full[s] (32 producer arrivals) and empty[s] (32 walker-warp
// arrivals); every wait is bounded by a clock deadline, after which the warp
// records an error (DevState.error) and leaves its loop.
// ---------------------------------------------------------------------------
constexpr int kRingSlots = 4;
// the ring, its full and empty barriers, and one 16-byte word that says which warp is the walker's
constexpr size_t kRingBytes = (size_t)kRingSlots * 32 * sizeof(PreTrial) + 2 * kRingSlots * sizeof(uint64_t) + 16;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Whole warp: waits until every lane has seen the phase with the given parity
// complete (each lane acquires for itself); false, for all lanes alike, once
// lane 0's clock passes the deadline.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* bar, uint32_t parity, long long deadline) {
  const uint32_t a = smem_addr(bar);
  bool ok = false;
  while (true) {
    if (!ok) ok = mbar_try_wait(a, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    if (__shfl_sync(0xffffffffu, clock64(), 0) > deadline) return false;
  }
}

// The draw of trial t of walker W, with the conflict mask of its group of 32
// (lane = t mod 32); the same values the in-kernel path computes.
template <int MODEL>
__device__ __forceinline__ PreTrial make_pretrial(const Problem& P, uint64_t t, int W, int lane) {
  const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
  int x, y;
  uint32_t pv;
  trial_site<MODEL>(P, r, x, y, pv);
  const float uf = __ull2float_rn(2ull * u52_bits(r.z, r.w) + 1ull) * 0x1p-53f;
  const int64_t thr = __float2ll_rn(logf(uf) * 1099511627776.0f);
  const uint32_t M = conflict_mask<MODEL, 32>(P, x, y, pv, lane, 0xffffffffu);
  return PreTrial{(uint32_t)x | ((uint32_t)y << 8) | (pv << 16), M, thr};
}

// Runs the sweeps of the nloc walkers wids[0..nloc) of one CTA (wpb walkers per CTA).
// RING: warp-specialised form (G = 32, one walker, 64 threads: one warp the
// walker, the other the producer of its draws).
template <int MODEL, int G, bool RING = false>
__device__ __forceinline__ void sweep_chain_body(const Problem& P, const DevState& S, uint32_t n_att, int wpb,
                                                 const int32_t* wids, int nloc, const PreTrial* pre = nullptr,
                                                 uint32_t pre_stride = 0,
                                                 long long wait_cycles = kDefaultWaitCycles) {
  static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32, "G");
  static_assert(!RING || G == 32, "the ring form runs one walker on one warp");
  // The sequential step skips the trials it need not visit (accepted for sure, energy unchanged)
  // when one walker owns the warp; with several walkers per warp the chains run in lockstep, the
  // longest decides, and the skip would cost more than it saves.
  constexpr bool kSkip = G == 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int wpad = P.w + 2 * kGuardBins;
  PreTrial* s_ring = reinterpret_cast<PreTrial*>(smem);                                  // [kRingSlots][32]
  uint64_t* s_full = reinterpret_cast<uint64_t*>(s_ring + kRingSlots * 32);              // [kRingSlots]
  uint64_t* s_empty = s_full + kRingSlots;                                               // [kRingSlots]
  int* s_swap = reinterpret_cast<int*>(s_empty + kRingSlots);                             // RING: 1 = roles swapped
  HotTrial* s_hot = reinterpret_cast<HotTrial*>(smem + (RING ? kRingBytes : 0));         // [G][wpb]
  ColdTrial* s_cold = reinterpret_cast<ColdTrial*>(s_hot + (G > 1 ? (size_t)wpb * G : 0));  // [G][wpb]
  int64_t* s_fx = reinterpret_cast<int64_t*>(s_cold + (G > 1 ? (size_t)wpb * G : 0));      // [wpad][wpb]
  uint32_t* s_lat = reinterpret_cast<uint32_t*>(s_fx + (size_t)wpad * wpb);
  uint32_t* s_J = s_lat + (size_t)P.lat_words * wpb;
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;

  for (int i = tid; i < nloc * wpad; i += nthr) {
    const int l = i / wpad, bp = i - l * wpad, b = bp - kGuardBins;
    int64_t v = 0;
    if (b >= 0 && b < P.w) v = to_fx(double_to_bits(S.lng[(size_t)wids[l] * P.w + b]));
    s_fx[bp * wpb + l] = v;
  }
  for (int i = tid; i < nloc * P.lat_words; i += nthr) {
    const int l = i / P.lat_words, j = i - l * P.lat_words;
    s_lat[j * wpb + l] = S.lat[(size_t)wids[l] * P.lat_words + j];
  }
  if (MODEL == kEA || MODEL == kEA3)
    for (int i = tid; i < P.j_words; i += nthr) s_J[i] = S.J[i];
  // RING: which warp of the CTA is the walker's.  An SM spreads its warps over its four
  // sub-partitions by hardware slot (%warpid mod 4), and a CTA of two warps takes two neighbouring
  // slots, so with several CTAs on one SM the first warps of all of them share the even
  // sub-partitions.  A CTA whose first slot lies in an odd group of four gives the walker to its
  // second warp, which spreads the chains over all four.  Only the placement depends on it: the
  // two roles compute the same whichever warp takes them.  rtid is the thread's index in its
  // role: [0, 32) the walker's warp, [32, 64) the producer.
  int rtid = tid;
  if constexpr (RING) {
    if (tid == 0) {
      uint32_t slot;
      asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
      *s_swap = (int)((slot >> 2) & 1u);
      for (int k = 0; k < kRingSlots; ++k) {
        mbar_init(&s_full[k], 32);
        mbar_init(&s_empty[k], 32);
      }
    }
    __syncthreads();
    if (*s_swap) rtid = tid ^ 32;
  } else {
    __syncthreads();
  }

  if (RING && rtid >= 32) {  // ---- producer warp
    if (nloc > 0) {
      const int W = wids[0];
      const uint64_t t0 = S.clock[0] * (uint64_t)P.N;
      const int lane = rtid - 32;
      const uint32_t n_groups = (n_att + 31) / 32;
      const long long deadline = __shfl_sync(0xffffffffu, clock64(), 0) + wait_cycles;
      for (uint32_t g = 0; g < n_groups; ++g) {
        const uint32_t sl = g % kRingSlots, rnd = g / kRingSlots;
        if (rnd >= 1 && !mbar_wait_warp(&s_empty[sl], (rnd - 1) & 1u, deadline)) {
          if (lane == 0) atomicOr(S.error, 1);
          break;
        }
        s_ring[sl * 32 + lane] = make_pretrial<MODEL>(P, t0 + (uint64_t)g * 32 + lane, W, lane);
        mbar_arrive(&s_full[sl]);
      }
    }
  }

  const int lw = rtid / G, lane = rtid % G;
  bool valid = lw < nloc && !(RING && rtid >= 32);
  int W = 0, a = 0, bin = 0, kexp = 0, wstart = 0;
  if (valid) {
    W = wids[lw];
    a = W / P.m;
    wstart = S.win_start[a];
    bin = (S.E[W] - P.e_min) / P.e_step - wstart;
    kexp = lnf_exponent(S.lnf[a]);
    if ((unsigned)bin >= (unsigned)window_width(P, S, a) || kexp == kBadLnf) {
      if (lane == 0) S.status[W] = kWalkerBadInput;
      valid = false;
    }
  }
  if (valid) {
    // 2^-39 <= ln f <= 64 (lnf_exponent): one visit adds 2^(40 - kexp) shadow units
    int64_t* fxp = s_fx + (size_t)kGuardBins * wpb + lw;  // fxp[b * wpb] = shadow of bin b, b in [-8, w+7]
    int64_t fx_cur = fxp[bin * wpb];
    uint64_t n_acc = 0, n_tie = 0, n_exact = 0;
    const uint32_t gm = group_mask<G>();
    const int w = window_width(P, S, a);  // the window test; P.w is the layout stride
    const uint64_t t0 = S.clock[0] * (uint64_t)P.N;
    HotTrial* my_hot = s_hot + lw;     // trial i of this walker's group: my_hot[i * wpb]
    ColdTrial* my_cold = s_cold + lw;

    const PreTrial* my_pre = pre ? pre + (size_t)W * pre_stride : nullptr;
    PreTrial nxt_pre{0u, 0u, 0};
    if (my_pre && (uint32_t)lane < n_att) nxt_pre = my_pre[lane];
    long long deadline = 0;
    if constexpr (RING) deadline = __shfl_sync(0xffffffffu, clock64(), 0) + wait_cycles;
    const int lsh = kFxBits - kexp;  // ln f = 2^-kexp is 2^lsh shadow units
    const int64_t lnf_fx = 1ll << lsh;
    for (uint32_t base = 0; base < n_att; base += G) {
      HotTrial tr;
      ColdTrial mv_own;  // this lane's move, written after the group if accepted
      uint32_t skipm = 0;  // trials of the group the sequential step skips (accepted, energy unchanged)
      {
        int x, y;
        uint32_t pv, M = 0;
        if constexpr (RING) {  // draw from the producer warp's ring
          const uint32_t g = base / 32, sl = g % kRingSlots;
          if (!mbar_wait_warp(&s_full[sl], (g / kRingSlots) & 1u, deadline)) {
            if (lane == 0) atomicOr(S.error, 2);
            break;  // uniform over the warp: every lane waits on the same phase
          }
          const PreTrial pt = s_ring[sl * 32 + lane];
          mbar_arrive(&s_empty[sl]);
          x = (int)(pt.pk & 0xffu);
          y = (int)((pt.pk >> 8) & 0xffu);
          pv = pt.pk >> 16;
          M = pt.mask;
          tr.thr = pt.thr;
        } else if (my_pre) {  // draw prepared ahead by k_precompute; prefetch the next group's
          const PreTrial pt = nxt_pre;
          if (base + G + (uint32_t)lane < n_att) nxt_pre = my_pre[base + G + lane];
          x = (int)(pt.pk & 0xffu);
          y = (int)((pt.pk >> 8) & 0xffu);
          pv = pt.pk >> 16;
          M = pt.mask;
          tr.thr = pt.thr;
        } else {
          const uint64_t t = t0 + base + (uint32_t)lane;
          const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
          trial_site<MODEL>(P, r, x, y, pv);
          const float uf = __ull2float_rn(2ull * u52_bits(r.z, r.w) + 1ull) * 0x1p-53f;
          tr.thr = __float2ll_rn(logf(uf) * 1099511627776.0f);
          if constexpr (G > 1) M = conflict_mask<MODEL, G>(P, x, y, pv, lane, gm);
        }
        const TrialEval<MODEL> ev = eval_trial<MODEL>(P, s_lat, s_J, wpb, lw, x, y, pv);
        tr.dbin = (int16_t)ev.dbin;
        tr.j = (uint16_t)lane;
        tr.mask = M;
        if constexpr (kSkip) tr.thr -= (int64_t)lane << lsh;  // the shadow clock of the group (below)
        mv_own.widx = ev.widx;
        mv_own.delta = ev.delta;
        mv_own.site = (uint32_t)x | ((uint32_t)y << 8) | (pv << 16);
        if constexpr (kSkip) {
          // A trial that leaves the energy unchanged is accepted (min[1, g/g] = 1) and stays in its
          // bin; when no earlier trial of the group touches its neighbourhood, that holds on the
          // configuration it will meet, so the sequential step need not visit it: it is skipped
          // (accepted, its ln f increment counted by the shadow clock), and the trials the step
          // does visit are staged in order, packed.
          const bool skip = ev.dbin == 0 && M == 0u;
          skipm = __ballot_sync(0xffffffffu, skip);
          if (!skip) my_hot[__popc(~skipm & ((1u << lane) - 1u)) * wpb] = tr;
          my_cold[lane * wpb] = mv_own;
        } else if constexpr (G > 1) {
          my_hot[lane * wpb] = tr;
          my_cold[lane * wpb] = mv_own;
        }
      }
      if constexpr (G > 1) __syncwarp(gm);

      uint32_t pending = 0;  // accepted trials of the group whose move is not written yet
      if (lane == 0) {
        // With the skip, the shadow clock: while the walker stays in one bin, its shadow grows by
        // ln f per trial, skipped or not.  fxa is the current bin's shadow minus (index in the
        // group) x ln f, so the shadow before trial j is fxa + j ln f; the staged threshold already
        // holds -j ln f, so the fast test reads fxa directly, and only a move needs j ln f.
        // Without it (several walkers per warp), fxa is the current bin's shadow itself.
        const int n_here = (int)min((uint32_t)G, n_att - base);
        const uint32_t valid = n_here >= 32 ? 0xffffffffu : ((1u << n_here) - 1u);
        const uint32_t skipv = skipm & valid;
        const int n_proc = __popc(valid & ~skipv);
        uint32_t accm = skipv, written = 0;
        int64_t fxa = fx_cur;
        if (n_proc > 0) {
          HotTrial cc = tr, cn = tr;  // the k-th and (k+1)-th visited trials
          if constexpr (G > 1) {
            cc = my_hot[0];
            cn = my_hot[(n_proc > 1 ? 1 : 0) * wpb];
          }
          int dj = cc.dbin;
          int64_t fxn = fxp[(bin + dj) * wpb];  // shadow of the first visited trial's target bin
          int k = 0;
          while (k < n_proc) {
            // ---- fast loop: no call and no large branch body inside; a trial that needs
            //      re-evaluation (conflict) or the exact test (band) leaves the loop
#pragma unroll 1
            for (; k < n_proc; ++k) {
              // loads that do not depend on this trial's outcome first (shared-memory operations
              // issue in order and must not queue behind this trial's stores)
              HotTrial cnn = cn;
              if constexpr (G > 1) cnn = my_hot[min(k + 2, n_proc - 1) * wpb];
              const int dn = cn.dbin;
              const int bn = bin + dj;
              const int64_t cand_stay = fxp[(bin + dn) * wpb];  // next visited trial's target if this one stays
              const int64_t cand_move = fxp[(bn + dn) * wpb];   // next visited trial's target if this one moves
              // accept iff (shadow_old - shadow_new) - ln u > guard; reject iff < -guard
              const bool inwin = (unsigned)bn < (unsigned)w;
              const int64_t lim_acc = fxa - cc.thr - kGuardFx;
              const int64_t lim_rej = fxa - cc.thr + kGuardFx;
              const bool acc = dj == 0 || (inwin && fxn < lim_acc);
              const bool band = dj != 0 && inwin && fxn >= lim_acc && fxn <= lim_rej;
              if (band || (accm & cc.mask) != 0u) break;
              const bool mv = acc && dj != 0;
              const int64_t jl = kSkip ? (int64_t)cc.j << lsh : 0;
              const int64_t fx_here = fxa + jl;           // the current bin's shadow before this trial
              if (mv) fxp[bin * wpb] = fx_here;           // write back the shadow of the bin left
              accm |= (uint32_t)acc << (kSkip ? (int)cc.j : k);
              const int64_t fwd = (dn == -dj) ? fx_here : cand_move;  // next target = the bin just left
              if constexpr (kSkip) fxa = mv ? fxn - jl : fxa;  // ln g(E) += ln f on the shadow (the clock)
              else fxa = (mv ? fxn : fxa) + lnf_fx;            // ln g(E) += ln f on the shadow
              fxn = mv ? fwd : cand_stay;
              bin = mv ? bn : bin;
              cc = cn;
              cn = cnn;
              dj = dn;
            }
            if (k >= n_proc) break;
            // ---- slow path for this trial: re-evaluate on the current configuration when an
            //      accepted earlier trial of the group touched its neighbourhood (first writing
            //      those moves), and decide exactly in FP64 when the fast test falls in the
            //      guard band
            const int j = kSkip ? (int)cc.j : k;
            const int64_t jl = kSkip ? (int64_t)j << lsh : 0;
            const int64_t fx_here = fxa + jl;
            const uint32_t hit = accm & cc.mask;
            TrialEval<MODEL> e2{};
            if (hit != 0u) {
              if constexpr (G > 1)
                for (uint32_t p = hit & ~written; p != 0u; p &= p - 1u) {
                  const ColdTrial c = my_cold[(__ffs(p) - 1) * wpb];
                  s_lat[c.widx] ^= c.delta;
                }
              written |= hit;
              const uint32_t site = G > 1 ? my_cold[j * wpb].site : mv_own.site;
              e2 = eval_trial<MODEL>(P, s_lat, s_J, wpb, lw, (int)(site & 0xffu), (int)((site >> 8) & 0xffu),
                                     site >> 16);
              dj = e2.dbin;
            }
            const int bn = bin + dj;
            const bool inwin = (unsigned)bn < (unsigned)w;
            fxn = fxp[bn * wpb];
            const int64_t dd = (fx_here - fxn) - (cc.thr + jl);
            bool acc = dj == 0 || (inwin && dd > kGuardFx);
            if (dj != 0 && inwin && dd >= -kGuardFx && dd <= kGuardFx) {
              const uint64_t t = t0 + base + (uint32_t)j;
              const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
              acc = exact_accept_fx(S, P, W, kexp, bin, fx_here, bn, fxn, u52_bits(r.z, r.w), n_tie);
              ++n_exact;
            }
            const bool mv = acc && dj != 0;
            if (acc && hit != 0u) {  // a re-evaluated move is written at once
              s_lat[e2.widx] ^= e2.delta;
              written |= 1u << j;
            }
            if (mv) fxp[bin * wpb] = fx_here;
            accm |= (uint32_t)acc << j;
            if constexpr (kSkip) fxa = mv ? fxn - jl : fxa;
            else fxa = (mv ? fxn : fxa) + lnf_fx;
            bin = mv ? bn : bin;
            ++k;
            if (k < n_proc) {  // re-prime the fast loop: the next two visited trials, and the next's target
              cc = cn;
              if constexpr (G > 1) cn = my_hot[min(k + 1, n_proc - 1) * wpb];
              dj = cc.dbin;
              fxn = fxp[(bin + dj) * wpb];
            }
          }
        }
        fx_cur = kSkip ? fxa + ((int64_t)n_here << lsh) : fxa;  // the shadow after the group's last trial
        n_acc += (uint64_t)__popc(accm);
        pending = accm & ~written;
      }
      // every lane writes its own trial's move if it was accepted and is not written yet; two such
      // moves never touch the same site (the later one would have met the earlier in its mask)
      if constexpr (G > 1) {
        pending = __shfl_sync(gm, pending, 0, G);
        if ((pending >> lane) & 1u) atomicXor(&s_lat[mv_own.widx], mv_own.delta);
        __syncwarp(gm);
      } else {
        if (pending & 1u) s_lat[mv_own.widx] ^= mv_own.delta;
      }
    }
    if (lane == 0) {
      fxp[bin * wpb] = fx_cur;
      S.E[W] = P.e_min + (wstart + bin) * P.e_step;
      S.wl_accept[W] += n_acc;
      S.near_ties[W] += n_tie;
      S.exact_tests[W] += n_exact;
    }
  }
  __syncthreads();

  // write back: visits = (shadow_end - shadow_start) / ln f; H += visits and the same number of
  // FP64 additions of ln f to ln g
  for (int i = tid; i < nloc * P.w; i += nthr) {
    const int l = i / P.w, b = i - l * P.w;
    const int Wl = wids[l];
    const size_t g = (size_t)Wl * P.w + b;
    const uint64_t v0 = double_to_bits(S.lng[g]);
    const int kx = lnf_exponent(S.lnf[Wl / P.m]);
    if (kx == kBadLnf) continue;  // a skipped walker: nothing ran
    const uint32_t c = (uint32_t)((s_fx[(b + kGuardBins) * wpb + l] - to_fx(v0)) >> (kFxBits - kx));
    if (c) {
      S.lng[g] = bits_to_double(add_pow2_repeated(v0, kx, c));
      S.H[g] += c;
    }
  }
  for (int i = tid; i < nloc * P.lat_words; i += nthr) {
    const int l = i / P.lat_words, j = i - l * P.lat_words;
    S.lat[(size_t)wids[l] * P.lat_words + j] = s_lat[j * wpb + l];
  }
}

template <int MODEL, int G>
__global__ void __launch_bounds__(256, 1) k_sweep_chain(Problem P, DevState S, SweepLaunch A) {
  const int first = blockIdx.x * A.wpb;
  sweep_chain_body<MODEL, G>(P, S, A.n_att, A.wpb, S.active + first, min(A.wpb, A.n_active - first), A.pre,
                             A.pre_stride);
}

// One walker per CTA of 64 threads (G = 32): one warp the walker, the other its draws.
template <int MODEL>
__global__ void __launch_bounds__(64, 1) k_sweep_ring(Problem P, DevState S, SweepLaunch A) {
  sweep_chain_body<MODEL, 32, true>(P, S, A.n_att, 1, S.active + blockIdx.x, 1, nullptr, 0, A.wait_cycles);
}

// ---------------------------------------------------------------------------
// Draws of the next sweep launch, prepared while the current one runs (on the
// SMs the walkers leave idle): for trial i of walker W the site, the proposed
// Potts offset, ln u, and the conflict mask of its group of G trials -- the
// same values the sweep kernel would compute, so the results are unchanged.
// One thread per (walker, trial) in a grid-stride loop over a small grid (one
// CTA per SM): a grid of thousands of CTAs that starts before the sweep
// kernel's CTAs are placed would hold the SMs and pack the walkers' CTAs onto
// few SMs when they free up.  Trials are padded to a multiple of 32, so every
// warp is wholly in range or wholly out of it.
// ---------------------------------------------------------------------------
template <int MODEL, int G>
__global__ void __launch_bounds__(256) k_precompute(Problem P, uint64_t t0, uint32_t n_att, uint32_t stride,
                                                    PreTrial* __restrict__ out) {
  const uint64_t total = (uint64_t)P.n_walkers * stride;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += step) {
    const int W = (int)(g / stride);
    const uint32_t i = (uint32_t)(g - (uint64_t)W * stride);
    const uint64_t t = t0 + i;
    const U4 r = philox10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, kTagFlip, P.seed_lo, P.seed_hi);
    int x, y;
    uint32_t pv;
    trial_site<MODEL>(P, r, x, y, pv);
    const float uf = __ull2float_rn(2ull * u52_bits(r.z, r.w) + 1ull) * 0x1p-53f;
    const int64_t thr = __float2ll_rn(logf(uf) * 1099511627776.0f);
    const uint32_t M = conflict_mask<MODEL, G>(P, x, y, pv, (int)(i % G), group_mask<G>());
    if (i < n_att) out[g] = PreTrial{(uint32_t)x | ((uint32_t)y << 8) | (pv << 16), M, thr};
  }
}

template <int MODEL>
static cudaError_t launch_precompute_m(int G, const Problem& P, uint64_t t0, uint32_t n_att, uint32_t stride,
                                       PreTrial* out, unsigned blocks, cudaStream_t st) {
  switch (G) {
    case 8: k_precompute<MODEL, 8><<<blocks, 256, 0, st>>>(P, t0, n_att, stride, out); break;
    case 16: k_precompute<MODEL, 16><<<blocks, 256, 0, st>>>(P, t0, n_att, stride, out); break;
    case 32: k_precompute<MODEL, 32><<<blocks, 256, 0, st>>>(P, t0, n_att, stride, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_precompute(int G, const Problem& P, uint64_t t0, uint32_t n_att, uint32_t stride, PreTrial* out,
                              int max_blocks, cudaStream_t st) {
  const uint64_t threads = (uint64_t)P.n_walkers * stride;
  const unsigned blocks = (unsigned)std::min<uint64_t>((threads + 255) / 256, (uint64_t)std::max(1, max_blocks));
  switch (P.model) {
    case kIsing: return launch_precompute_m<kIsing>(G, P, t0, n_att, stride, out, blocks, st);
    case kPotts: return launch_precompute_m<kPotts>(G, P, t0, n_att, stride, out, blocks, st);
    case kEA: return launch_precompute_m<kEA>(G, P, t0, n_att, stride, out, blocks, st);
    case kEA3: return launch_precompute_m<kEA3>(G, P, t0, n_att, stride, out, blocks, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Replica exchange, Eq. (1).  One CTA per window pair (a, a+1), a = round
// (mod 2); walker k of window a is paired with walker sigma(k) of window a+1,
// sigma a Fisher-Yates permutation from the round's own stream.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void exchange_body(const Problem& P, const DevState& S, int pair_block) {
  extern __shared__ int sigma[];
  const uint32_t round = (uint32_t)S.clock[1];
  const int a = 2 * pair_block + (int)(round & 1u);
  if (a + 1 >= P.h) return;
  if (S.done[a] || S.done[a + 1]) return;
  const int m = P.m;
  if (threadIdx.x == 0) {
    for (int k = 0; k < m; ++k) sigma[k] = k;
    for (int i = m - 1; i >= 1; --i) {
      const U4 r = philox10(round, (uint32_t)a, (uint32_t)i, kTagPerm, P.seed_lo, P.seed_hi);
      const int j = (int)scale32(r.x, (uint32_t)(i + 1));
      const int tmp = sigma[i];
      sigma[i] = sigma[j];
      sigma[j] = tmp;
    }
  }
  __syncthreads();
  const int loA = P.e_min + S.win_start[a] * P.e_step, hiA = loA + (window_width(P, S, a) - 1) * P.e_step;
  const int loB = P.e_min + S.win_start[a + 1] * P.e_step, hiB = loB + (window_width(P, S, a + 1) - 1) * P.e_step;
  unsigned n_acc = 0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int Wi = a * m + k, Wj = (a + 1) * m + sigma[k];
    const int EX = S.E[Wi], EY = S.E[Wj];
    if (EX < loB || EX > hiB || EY < loA || EY > hiA) continue;
    const double* gi = S.lng + (size_t)Wi * P.w;
    const double* gj = S.lng + (size_t)Wj * P.w;
    const int iX = (EX - loA) / P.e_step, iY = (EY - loA) / P.e_step;
    const int jX = (EX - loB) / P.e_step, jY = (EY - loB) / P.e_step;
    const double d1 = __dsub_rn(gi[iX], gi[iY]);
    const double d2 = __dsub_rn(gj[jY], gj[jX]);
    const double D = __dadd_rn(d1, d2);
    bool acc = D >= 0.0;
    if (!acc) {
      const U4 r = philox10(round, (uint32_t)a, (uint32_t)k, kTagXacc, P.seed_lo, P.seed_hi);
      const double u = __dmul_rn(__ull2double_rn(2ull * u52_bits(r.z, r.w) + 1ull), 0x1p-53);
      const double lu = log(u);
      if (fabs(__dsub_rn(lu, D)) < 1e-12) S.near_ties[Wi] += 1;
      acc = lu < D;
    }
    if (acc) {
      uint32_t* li = S.lat + (size_t)Wi * P.lat_words;
      uint32_t* lj = S.lat + (size_t)Wj * P.lat_words;
      for (int i = 0; i < P.lat_words; ++i) {
        const uint32_t t = li[i];
        li[i] = lj[i];
        lj[i] = t;
      }
      S.E[Wi] = EY;
      S.E[Wj] = EX;
      ++n_acc;
      if (S.rep_id) {  // the replicas travel with their configurations
        const int32_t ri = S.rep_id[Wj], rj = S.rep_id[Wi];
        S.rep_id[Wi] = ri;
        S.rep_id[Wj] = rj;
        if (a == 0) {  // ri arrives in the lowest window
          if (S.rep_state[ri] == 2) S.rep_trips[ri] += 1;
          S.rep_state[ri] = 1;
        }
        if (a + 1 == P.h - 1 && S.rep_state[rj] == 1) S.rep_state[rj] = 2;  // rj reaches the highest
      }
    }
  }
  if (n_acc) atomicAdd(reinterpret_cast<unsigned long long*>(&S.x_accepted[a]), (unsigned long long)n_acc);
  if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&S.x_tried[a]), (unsigned long long)m);
}

__global__ void k_exchange(Problem P, DevState S) { exchange_body(P, S, (int)blockIdx.x); }

// ---------------------------------------------------------------------------
// Flatness, merge and f update.  One CTA per window.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flat_merge_body(const Problem& P, const DevState& S, int a) {
  if (S.done[a]) return;
  __shared__ uint32_t r_min[32];
  __shared__ unsigned long long r_sum[32];
  __shared__ int r_n[32];
  __shared__ int all_flat;
  const int m = P.m, w = window_width(P, S, a), ld = P.w;  // window bins; row stride
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  // 1/t rule: ln f = 2^-k; t >= 2^(k+1) trials per level iff clock * N >= w * 2^(k+1)
  const int k = 1023 - (int)((double_to_bits(S.lnf[a]) >> 52) & 0x7FF);
  const uint64_t trials = S.clock[0] * (uint64_t)P.N;
  const uint64_t next = k + 1 < 48 ? (uint64_t)w << (k + 1) : ~0ull;
  const int stage = P.wl_rule == 1 ? S.stage[a] : 0;
  if (threadIdx.x == 0) all_flat = 1;
  __syncthreads();
  if (stage == 1) {
    if (trials < next) return;  // uniform: t has not reached 2^(k+1)
  } else {
    for (int kw = 0; kw < m; ++kw) {
      const int W = a * m + kw;
      uint32_t hmin = 0xffffffffu;
      unsigned long long sum = 0;
      int n = 0;
      for (int b = threadIdx.x; b < w; b += blockDim.x) {
        if (S.lng[(size_t)W * ld + b] > 0.0) {
          const uint32_t hv = S.H[(size_t)W * ld + b];
          hmin = min(hmin, hv);
          sum += hv;
          ++n;
        }
      }
      for (int o = 16; o; o >>= 1) {
        hmin = min(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
      }
      if (lane == 0) {
        r_min[wid] = hmin;
        r_sum[wid] = sum;
        r_n[wid] = n;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t hm = 0xffffffffu;
        unsigned long long ss = 0;
        int nn = 0;
        for (int i = 0; i < nw; ++i) {
          hm = min(hm, r_min[i]);
          ss += r_sum[i];
          nn += r_n[i];
        }
        // flatness rule: min H * n >= flatness * sum H over the visited bins;
        // 1/t rule, first stage: every visited bin seen again (min H > 0)
        const bool ok = P.wl_rule == 1 ? (nn > 0 && hm > 0u)
                                       : (nn > 0 && __dmul_rn(__uint2double_rn(hm), __int2double_rn(nn)) >=
                                                        __dmul_rn(P.flatness, __ull2double_rn(ss)));
        if (!ok) all_flat = 0;
      }
      __syncthreads();
      if (!all_flat) return;
    }
  }
  // merge: mean of the m estimators (summed in walker order), H reset
  for (int b = threadIdx.x; b < w; b += blockDim.x) {
    double sum = S.lng[(size_t)(a * m) * ld + b];
    for (int kw = 1; kw < m; ++kw) sum = __dadd_rn(sum, S.lng[(size_t)(a * m + kw) * ld + b]);
    const double mean = __ddiv_rn(sum, (double)m);
    for (int kw = 0; kw < m; ++kw) {
      S.lng[(size_t)(a * m + kw) * ld + b] = mean;
      S.H[(size_t)(a * m + kw) * ld + b] = 0u;
    }
  }
  if (threadIdx.x == 0) {
    if (S.iter[a] == 0 && S.first_iter) S.first_iter[a] = (int64_t)S.clock[0];  // end of the first iteration
    S.iter[a] += 1;
    if (P.wl_rule == 1 && stage == 0 && trials < next) {
      S.stage[a] = 1;  // halving would take ln f below 1/t: follow 1/t from here
    } else {
      const double lnf = __dmul_rn(S.lnf[a], 0.5);  // f -> sqrt(f)
      S.lnf[a] = lnf;
      if (lnf < P.lnf_final) {
        S.done[a] = 1;
        atomicAdd(S.n_done, 1);
      }
    }
  }
}

__global__ void k_flat_merge(Problem P, DevState S) { flat_merge_body(P, S, (int)blockIdx.x); }

// ---------------------------------------------------------------------------
// Served form: the same phase bodies over many request slots in one launch.
// Sweep: one CTA per (slot, walker) of the model's walker list, G = 32.
// Exchange: one CTA per (slot, window pair).  Clock: one thread per slot.
// Flatness: one CTA per (slot, window), acting only on slots whose sweep
// clock is at a multiple of their flatness period.  Every request keeps its
// own schedule, streams and state, so its trajectory is the one it has alone.
// ---------------------------------------------------------------------------
// A shape group holds one model, so each form is instantiated per model and
// the group's launch picks the one of its model.  One walker per 32-lane CTA:
template <int MODEL>
__global__ void __launch_bounds__(32, 16) k_sweep_batch(const BatchSlot* __restrict__ slots,
                                                        const BatchWalker* __restrict__ list) {
  __shared__ int32_t wid;
  const BatchWalker bw = list[blockIdx.x];
  const Problem P = slots[bw.slot].P;
  const DevState S = slots[bw.slot].S;
  const uint32_t n_att = slots[bw.slot].n_att;
  if (!slots[bw.slot].active || S.done[bw.W / P.m]) return;  // uniform over the CTA
  if (threadIdx.x == 0) wid = bw.W;
  __syncthreads();
  sweep_chain_body<MODEL, 32>(P, S, n_att, 1, &wid, 1);
}

// The same with a producer warp per walker (the ring form): for rounds with few
// walkers on the GPU, where each walker's chain has an SM sub-partition of its own.
template <int MODEL>
__global__ void __launch_bounds__(64, 8) k_sweep_batch_ring(const BatchSlot* __restrict__ slots,
                                                            const BatchWalker* __restrict__ list) {
  __shared__ int32_t wid;
  const BatchWalker bw = list[blockIdx.x];
  const Problem P = slots[bw.slot].P;
  const DevState S = slots[bw.slot].S;
  const uint32_t n_att = slots[bw.slot].n_att;
  if (!slots[bw.slot].active || S.done[bw.W / P.m]) return;  // uniform over the CTA
  if (threadIdx.x == 0) wid = bw.W;
  __syncthreads();
  sweep_chain_body<MODEL, 32, true>(P, S, n_att, 1, &wid, 1);
}

// For rounds with many walkers on the GPU (the chains share the SMs and the
// issue slots are what runs out): up to 4 walkers of one request per CTA, 8
// lanes each, so that one instruction of the sequential step serves 4 chains.
// Entry (slot, W0) covers walkers W0 .. W0+3 of the slot; walkers of finished
// windows are left out.
template <int MODEL>
__global__ void __launch_bounds__(32, 16) k_sweep_batch_quad(const BatchSlot* __restrict__ slots,
                                                             const BatchWalker* __restrict__ list) {
  __shared__ int32_t wids[4];
  __shared__ int32_t nloc;
  const BatchWalker bw = list[blockIdx.x];
  const Problem P = slots[bw.slot].P;
  const DevState S = slots[bw.slot].S;
  const uint32_t n_att = slots[bw.slot].n_att;
  if (!slots[bw.slot].active) return;  // uniform over the CTA
  if (threadIdx.x == 0) {
    int n = 0;
    for (int W = bw.W; W < bw.W + 4 && W < P.n_walkers; ++W)
      if (!S.done[W / P.m]) wids[n++] = W;
    nloc = n;
  }
  __syncthreads();
  if (nloc == 0) return;  // uniform over the CTA
  sweep_chain_body<MODEL, 8>(P, S, n_att, 4, wids, nloc);
}

__global__ void k_exchange_batch(const BatchSlot* __restrict__ slots, int max_pairs) {
  const int s = (int)blockIdx.x / max_pairs, p = (int)blockIdx.x % max_pairs;
  if (!slots[s].active) return;
  const Problem P = slots[s].P;
  const DevState S = slots[s].S;
  exchange_body(P, S, p);
}

__global__ void k_advance_batch(const BatchSlot* __restrict__ slots, int n_slots) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots || !slots[s].active) return;
  const int h = slots[s].P.h, nd = *slots[s].S.n_done;  // windows done before this round's check
  if (nd >= h) return;                                   // finished: the clocks stay
  uint64_t* clk = slots[s].S.clock;
  clk[0] += slots[s].spe;
  clk[1] += 1;
  clk[2] += (uint64_t)(h - nd) * (uint64_t)slots[s].P.m * slots[s].n_att;
}

__global__ void k_flat_batch(const BatchSlot* __restrict__ slots, int max_h) {
  const int s = (int)blockIdx.x / max_h, a = (int)blockIdx.x % max_h;
  if (!slots[s].active || a >= slots[s].P.h) return;
  if (slots[s].S.clock[0] % slots[s].spf != 0) return;
  const Problem P = slots[s].P;
  const DevState S = slots[s].S;
  flat_merge_body(P, S, a);
}

// Copies every slot's count of finished windows and its clocks into one array.
__global__ void k_slot_report(const BatchSlot* __restrict__ slots, int n_slots, SlotReport* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  SlotReport r{-1, 0, 0, 0, 0};
  if (slots[s].active) {
    const uint64_t* clk = slots[s].S.clock;
    r = SlotReport{*slots[s].S.n_done, 1, clk[0], clk[1], clk[2]};
  }
  out[s] = r;
}

// k_sweep_batch has a few bytes of static shared memory, so its dynamic
// allowance stays below the 227 KB per-CTA limit.
constexpr int kBatchDynSmem = 226 * 1024;

size_t ring_extra_smem() { return kRingBytes; }
size_t batch_smem_limit() { return kBatchDynSmem; }

template <int MODEL>
static cudaError_t prepare_sweep_batch_m() {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_batch<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchDynSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_sweep_batch_quad<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchDynSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_sweep_batch_ring<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchDynSmem);
}

cudaError_t prepare_sweep_batch() {
  cudaError_t e = prepare_sweep_batch_m<kIsing>();
  if (e == cudaSuccess) e = prepare_sweep_batch_m<kPotts>();
  if (e == cudaSuccess) e = prepare_sweep_batch_m<kEA>();
  if (e == cudaSuccess) e = prepare_sweep_batch_m<kEA3>();
  return e;
}

template <int MODEL>
static void launch_sweep_batch_m(const BatchSlot* d_slots, const BatchWalker* d_list, int n_list, size_t smem,
                                 int form, cudaStream_t st) {
  if (form == kBatchRing) k_sweep_batch_ring<MODEL><<<n_list, 64, smem + kRingBytes, st>>>(d_slots, d_list);
  else if (form == kBatchQuad) k_sweep_batch_quad<MODEL><<<n_list, 32, smem, st>>>(d_slots, d_list);
  else k_sweep_batch<MODEL><<<n_list, 32, smem, st>>>(d_slots, d_list);
}

cudaError_t launch_round_batch(const BatchSlot* d_slots, int n_slots, const BatchWalker* d_list, int n_list,
                               size_t smem, int max_pairs, int max_m, int max_h, int form, int model,
                               cudaStream_t st) {
  if (n_list > 0) {
    switch (model) {
      case kIsing: launch_sweep_batch_m<kIsing>(d_slots, d_list, n_list, smem, form, st); break;
      case kPotts: launch_sweep_batch_m<kPotts>(d_slots, d_list, n_list, smem, form, st); break;
      case kEA: launch_sweep_batch_m<kEA>(d_slots, d_list, n_list, smem, form, st); break;
      case kEA3: launch_sweep_batch_m<kEA3>(d_slots, d_list, n_list, smem, form, st); break;
      default: return cudaErrorInvalidValue;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (max_pairs > 0) {
    const int threads = max_m < 128 ? ((max_m + 31) / 32) * 32 : 128;
    k_exchange_batch<<<n_slots * max_pairs, threads, (size_t)max_m * sizeof(int), st>>>(d_slots, max_pairs);
  }
  k_advance_batch<<<(n_slots + 127) / 128, 128, 0, st>>>(d_slots, n_slots);
  k_flat_batch<<<n_slots * max_h, 256, 0, st>>>(d_slots, max_h);
  return cudaGetLastError();
}

cudaError_t launch_slot_report(const BatchSlot* d_slots, int n_slots, SlotReport* out, cudaStream_t st) {
  if (n_slots <= 0) return cudaSuccess;
  k_slot_report<<<(n_slots + 127) / 128, 128, 0, st>>>(d_slots, n_slots, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
// G <= 4 lanes per walker: k_sweep; G >= 8: the speculative k_sweep_spec.
template <int MODEL, int G>
static auto sweep_kernel(int variant) {
  return variant == kSweepStaged ? k_sweep_spec<MODEL, G> : k_sweep_chain<MODEL, G>;
}

template <int MODEL, int G>
static cudaError_t prepare_sweep_t() {
  cudaError_t e = cudaFuncSetAttribute(k_sweep_spec<MODEL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  if (G == 32) {
    e = cudaFuncSetAttribute(k_sweep_ring<MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_sweep_chain<MODEL, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

template <int MODEL>
static cudaError_t prepare_sweep_m(int G) {
  switch (G) {
    case 1: return prepare_sweep_t<MODEL, 1>();
    case 2: return prepare_sweep_t<MODEL, 2>();
    case 4: return prepare_sweep_t<MODEL, 4>();
    case 8: return prepare_sweep_t<MODEL, 8>();
    case 16: return prepare_sweep_t<MODEL, 16>();
    case 32: return prepare_sweep_t<MODEL, 32>();
  }
  return cudaErrorInvalidValue;
}

// Allows the sweep kernel of (model, G) up to 227 KB of dynamic shared memory.
cudaError_t prepare_sweep(int G, int model) {
  switch (model) {
    case kIsing: return prepare_sweep_m<kIsing>(G);
    case kPotts: return prepare_sweep_m<kPotts>(G);
    case kEA: return prepare_sweep_m<kEA>(G);
    case kEA3: return prepare_sweep_m<kEA3>(G);
  }
  return cudaErrorInvalidValue;
}

template <int MODEL, int G>
static cudaError_t launch_sweep_t(const Problem& P, const DevState& S, const SweepLaunch& A, size_t smem,
                                  cudaStream_t st) {
  if (A.variant == kSweepRing) {  // one walker per CTA: its warp and a producer warp
    if (G != 32 || A.wpb != 1) return cudaErrorInvalidValue;
    k_sweep_ring<MODEL><<<A.n_active, 64, smem, st>>>(P, S, A);
    return cudaGetLastError();
  }
  const int blocks = (A.n_active + A.wpb - 1) / A.wpb;
  sweep_kernel<MODEL, G>(A.variant)<<<blocks, A.wpb * G, smem, st>>>(P, S, A);
  return cudaGetLastError();
}

template <int MODEL>
static cudaError_t launch_sweep_m(int G, const Problem& P, const DevState& S, const SweepLaunch& A, size_t smem,
                                  cudaStream_t st) {
  switch (G) {
    case 1: return launch_sweep_t<MODEL, 1>(P, S, A, smem, st);
    case 2: return launch_sweep_t<MODEL, 2>(P, S, A, smem, st);
    case 4: return launch_sweep_t<MODEL, 4>(P, S, A, smem, st);
    case 8: return launch_sweep_t<MODEL, 8>(P, S, A, smem, st);
    case 16: return launch_sweep_t<MODEL, 16>(P, S, A, smem, st);
    case 32: return launch_sweep_t<MODEL, 32>(P, S, A, smem, st);
  }
  return cudaErrorInvalidValue;
}

size_t sweep_smem_bytes(const Problem& P, int wpb, int G, int variant) {
  size_t b = variant == kSweepStaged ? (size_t)wpb * ((size_t)P.w * 12 + (size_t)P.lat_words * 4)
                                     : (size_t)wpb * ((size_t)(P.w + 2 * kGuardBins) * 8 + (size_t)P.lat_words * 4);
  if (G > 1) b += (size_t)wpb * G * (variant == kSweepStaged ? sizeof(StagedTrial) : kChainStagingBytes);
  if (P.model == kEA || P.model == kEA3) b += (size_t)P.j_words * 4;
  if (variant == kSweepRing) b += kRingBytes;
  return b;
}

cudaError_t launch_sweep(int G, const Problem& P, const DevState& S, const SweepLaunch& A, cudaStream_t st) {
  if (A.n_active <= 0) return cudaSuccess;
  const size_t smem = sweep_smem_bytes(P, A.wpb, G, A.variant);
  switch (P.model) {
    case kIsing: return launch_sweep_m<kIsing>(G, P, S, A, smem, st);
    case kPotts: return launch_sweep_m<kPotts>(G, P, S, A, smem, st);
    case kEA: return launch_sweep_m<kEA>(G, P, S, A, smem, st);
    case kEA3: return launch_sweep_m<kEA3>(G, P, S, A, smem, st);
  }
  return cudaErrorInvalidValue;
}

// One CTA per possible pair of either parity; CTAs of the other parity exit.
cudaError_t launch_exchange(const Problem& P, const DevState& S, cudaStream_t st) {
  const int pairs = P.h / 2;
  if (pairs <= 0) return cudaSuccess;
  const int threads = P.m < 128 ? ((P.m + 31) / 32) * 32 : 128;
  k_exchange<<<pairs, threads, (size_t)P.m * sizeof(int), st>>>(P, S);
  return cudaGetLastError();
}

__global__ void k_advance_clock(DevState S, uint32_t sweeps) {
  S.clock[0] += sweeps;
  S.clock[1] += 1;
}

cudaError_t launch_advance_clock(const DevState& S, uint32_t sweeps, cudaStream_t st) {
  k_advance_clock<<<1, 1, 0, st>>>(S, sweeps);
  return cudaGetLastError();
}

cudaError_t launch_flat_merge(const Problem& P, const DevState& S, cudaStream_t st) {
  k_flat_merge<<<P.h, 256, 0, st>>>(P, S);
  return cudaGetLastError();
}

cudaError_t launch_init(const Problem& P, const DevState& S, cudaStream_t st) {
  k_init_lattice<<<(P.n_walkers + 63) / 64, 64, 0, st>>>(P, S);
  return cudaGetLastError();
}

cudaError_t launch_descent(const Problem& P, const DevState& S, uint64_t n_att, cudaStream_t st) {
  k_descent<<<(P.n_walkers + 63) / 64, 64, 0, st>>>(P, S, n_att);
  return cudaGetLastError();
}

cudaError_t launch_entry(const Problem& P, const DevState& S, uint64_t budget, cudaStream_t st) {
  k_entry<<<(P.n_walkers + 63) / 64, 64, 0, st>>>(P, S, budget);
  return cudaGetLastError();
}

}  // namespace rewl
