// rewl_device.cuh -- device-side building blocks of the REWL library:
// the Philox4x32-10 generator, the lattice bit layout, the exact integer
// emulation of ln g += ln f, and the fixed-point shadow of ln g used by the
// WL acceptance test.
#pragma once
#include <cstdint>

#include "rewl_layout.h"

namespace rewl {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplications with the round key bumped by the Weyl constants.
// Host and device share this definition inside the library.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = mulhi32(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = mulhi32(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  return U4{c0, c1, c2, c3};
}

// floor(r * n / 2^32)
__host__ __device__ __forceinline__ uint32_t scale32(uint32_t r, uint32_t n) { return mulhi32(r, n); }

// 52 random bits k from two words; u = (2k+1) 2^-53 lies in (0, 1).
__host__ __device__ __forceinline__ uint64_t u52_bits(uint32_t r2, uint32_t r3) {
  return ((uint64_t)r2 << 20) | (uint64_t)(r3 >> 12);
}

// ---------------------------------------------------------------------------
// Exact FP64 arithmetic on non-negative ln g values without the FP64 pipe.
// ---------------------------------------------------------------------------
constexpr uint64_t kFracMask = (1ull << 52) - 1;

__device__ __forceinline__ double bits_to_double(uint64_t b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ uint64_t double_to_bits(double d) { return (uint64_t)__double_as_longlong(d); }

// V (bits of a double >= 0) plus c successive IEEE additions of 2^-k, exactly
// as c separate round-to-nearest FP64 additions would produce it.  While the
// sum stays inside V's binade every addition is exact and moves the fraction
// field by 2^(52-e-k) units; the (rare) additions that cross into the next
// binade, or where 2^-k is not a whole number of V's ulps, are done by the
// FP64 unit itself.
__device__ __forceinline__ uint64_t pow2_bits(int k) { return (uint64_t)(1023 - k) << 52; }  // bits of 2^-k

static __device__ __noinline__ uint64_t add_pow2_repeated(uint64_t V, int k, uint32_t c) {
  const double inc_d = bits_to_double(pow2_bits(k));
  while (c > 0) {
    if (V == 0) {
      V = pow2_bits(k);
      --c;
      continue;
    }
    const int e = (int)((V >> 52) & 0x7FF) - 1023;
    const int sh = 52 - e - k;
    if (sh < 0 || sh > 52) {
      V = double_to_bits(__dadd_rn(bits_to_double(V), inc_d));
      --c;
      continue;
    }
    const uint64_t room = (kFracMask - (V & kFracMask)) >> sh;
    if ((uint64_t)c <= room) {
      V += (uint64_t)c << sh;
      c = 0;
    } else {
      V += room << sh;
      c -= (uint32_t)room;
      V = double_to_bits(__dadd_rn(bits_to_double(V), inc_d));
      --c;
    }
  }
  return V;
}

// Fixed-point shadow: floor(v * 2^40) of a double v >= 0 given by its bits
// (exact for the integer part, truncation error < 2^-40).
constexpr int kFxBits = 40;
__device__ __forceinline__ int64_t to_fx(uint64_t V) {
  if (V == 0) return 0;
  const int e = (int)((V >> 52) & 0x7FF) - 1023;
  const uint64_t M = (V & kFracMask) | (1ull << 52);
  const int s = e - (52 - kFxBits);  // fx = M * 2^(e - 12)
  if (s >= 0) return (int64_t)(M << s);
  if (s <= -64) return 0;
  return (int64_t)(M >> (-s));
}

// ln f of a window as the exponent k of ln f = 2^-k, or kBadLnf when ln f is
// not a power of two with -6 <= k <= 39 (the range the shadow's increment
// 2^(40-k) and the exact repeated additions of ln g are written for; the
// library's own windows always satisfy it: ln f0 <= 64, ln f_final >= 1e-12).
constexpr int kBadLnf = -1000;
__device__ __forceinline__ int lnf_exponent(double lnf) {
  const uint64_t b = double_to_bits(lnf);
  const int k = 1023 - (int)((b >> 52) & 0x7FF);
  if ((b & ~(0x7FFull << 52)) != 0 || k < -6 || k > kFxBits - 1) return kBadLnf;  // sign, mantissa or range
  return k;
}

// Per-walker status a sweep kernel leaves in DevState.status for a walker it
// skipped (a walker is skipped only on inputs the library itself never makes).
enum WalkerStatus : int32_t { kWalkerOk = 0, kWalkerBadInput = 1 };

// Guard band of the fast acceptance test, in units of 2^-40: 2^24 units =
// 1.5e-5 covers |logf(u) - ln u| <= 1 ulp(float) + float rounding of u
// (< 4e-6 for ln u > -37) plus the shadow's truncation (< 1e-11).
constexpr int64_t kGuardFx = 1ll << 24;

// ---------------------------------------------------------------------------
// Packed lattice access.  Ising / +-J: 1 bit per site, row y holds Wr 32-bit
// words, site (x, y) is bit (x & 31) of word x >> 5.  Potts: 4 bits per site,
// site (x, y) is nibble (x & 7) of word x >> 3.  SMEM copies interleave
// walkers: word j of local walker lw is at s[j * wpb + lw].
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t spin_bit(const uint32_t* s, int wpb, int lw, int Wr, int x, int y) {
  return (s[(y * Wr + (x >> 5)) * wpb + lw] >> (x & 31)) & 1u;
}
__device__ __forceinline__ uint32_t potts_val(const uint32_t* s, int wpb, int lw, int Wr, int x, int y) {
  return (s[(y * Wr + (x >> 3)) * wpb + lw] >> ((x & 7) * 4)) & 15u;
}
__device__ __forceinline__ uint32_t coupling_bit(const uint32_t* J, int Wr1, int plane, int L, int x, int y) {
  return (J[(plane * L + y) * Wr1 + (x >> 5)] >> (x & 31)) & 1u;
}

}  // namespace rewl
