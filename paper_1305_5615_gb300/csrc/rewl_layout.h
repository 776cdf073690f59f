// rewl_layout.h -- device data layout and kernel arguments of one REWL solve.
//
// HBM layout (all walker-major; walker W = a*m + k is walker k of window a):
//   lat   u32 [n_walkers][lat_words]   packed configurations
//   E     i32 [n_walkers]              current energies
//   lng   f64 [n_walkers][w]           ln g over the window's w bins
//   H     u32 [n_walkers][w]           visit histogram of the iteration
//   J     u32 [dim][rows][Wr1]         +-J couplings, bit 1 = J -1 (planes: right, down[, behind])
//   win_start i32 [h], win_width i32 [h] (P.w = the largest, the row stride of lng and H),
//   lnf f64 [h], iter i32 [h], done i32 [h], stage i32 [h], first_iter i64 [h]
//   counters u64: wl_accept / near_ties / exact_tests [n_walkers], x_tried / x_accepted [h]
#pragma once
#include <cstdint>

namespace rewl {

enum Model : int { kIsing = 0, kPotts = 1, kEA = 2, kEA3 = 3 };  // kEA3: +-J on the L x L x L cube
// 4th Philox counter word: one stream per purpose.
enum Tag : uint32_t { kTagFlip = 0, kTagEntry = 1, kTagPerm = 2, kTagXacc = 3, kTagInit = 4, kTagCoupling = 5 };

struct Problem {
  int model, q, L, N;
  int rows;        // lattice rows: L (2D), L * L (3D: row = z * L + y)
  int Wr;          // words per lattice row (1-bit or 4-bit sites)
  int Wr1;         // words per row of a coupling plane
  int lat_words;   // rows * Wr
  int j_words;     // coupling words: dim planes (right, down[, behind]) of rows * Wr1
  int e_min, e_step, n_bins;
  int h, m, w, n_walkers;
  uint32_t magic_L;   // ceil(2^32 / L): y = mulhi(site, magic_L) for site < L^2 (2D)
  uint32_t magic_L2;  // ceil(2^32 / L^2): z = mulhi(site, magic_L2) for site < L^3 (3D)
  uint32_t seed_lo, seed_hi;
  int wl_rule;     // 0: flatness rule; 1: 1/t rule
  double flatness, lnf_final;
};

struct DevState {
  uint32_t* lat;
  uint32_t* J;
  int32_t* E;
  double* lng;
  uint32_t* H;
  int32_t* win_start;
  double* lnf;
  int32_t* iter;
  int32_t* done;
  int32_t* n_done;
  uint64_t* wl_accept;
  uint64_t* near_ties;
  uint64_t* exact_tests;
  uint64_t* x_tried;
  uint64_t* x_accepted;
  int32_t* active;       // walker ids the sweep kernel runs, in order
  int32_t* status;       // per walker: 0 ok, else a rewl_status
  uint64_t* entry_t;     // per walker counter of the entry stream
  uint32_t* seed_config; // restart configuration for the entry walk
  uint64_t* clock;       // [0] sweeps done by the solve, [1] exchange rounds done, [2] trials (batched rounds)
  int32_t* stage;        // [h] 1/t rule: 0 = halving on the histogram test, 1 = following 1/t
  int32_t* win_width;    // [h] bins of each window (NULL: P.w for all)
  int64_t* first_iter;   // [h] sweep clock of each window's first merge, -1 before (may be NULL)
  int32_t* error;        // one word: bits set by a sweep kernel whose bounded wait ran out (may be NULL)
  // replica round trips (Fig. 3): rep_id[W] = the replica (configuration) walker W holds;
  // per replica: rep_state 0 = not yet in the lowest window, 1 = has been there, 2 = has since
  // reached the highest window; rep_trips = completed lowest -> highest -> lowest trips
  int32_t* rep_id;
  int32_t* rep_state;
  int64_t* rep_trips;
};

// Sweep kernel variants (identical results): the staged form keeps H in
// shared memory and runs a one-deep sequential chain; the chain form
// speculates two deep and rebuilds H from the shadow; the ring form is the
// chain form with the draws made by a second, producer warp.
enum SweepVariant : int { kSweepChain = 0, kSweepStaged = 1, kSweepRing = 2 };

// A trial's draw, prepared ahead of its sweep launch by k_precompute: the
// site (x | y << 8), the proposed Potts offset (<< 16), the mask of earlier
// trials of its group that touch its neighbourhood, and ln u in 2^-40 units.
struct PreTrial {
  uint32_t pk;
  uint32_t mask;
  int64_t thr;
};

// Default bound of the ring form's hand-off waits (SM clock cycles from the
// start of a sweep launch): about 8 s at 2 GHz, while a launch takes milliseconds.
constexpr long long kDefaultWaitCycles = 1ll << 34;

struct SweepLaunch {
  uint32_t n_att;     // trials per walker in this launch (sweeps * N); the first
                      // trial's index is clock[0] * N, read on the device
  int n_active;       // walkers in `active`
  int wpb;            // walkers per CTA
  int variant;        // SweepVariant
  const PreTrial* pre;  // prepared draws [walker][pre_stride] or nullptr (drawn in the kernel)
  uint32_t pre_stride;
  long long wait_cycles;  // ring form: bound of the hand-off waits (kDefaultWaitCycles)
};

// One request slot of the served form: the request's sizes and device
// arrays, as used by its own single-solve kernels.
struct BatchSlot {
  Problem P;
  DevState S;
  uint32_t n_att;   // trials per walker per block: sweeps_per_exchange * N
  uint32_t spe;     // sweeps_per_exchange
  uint32_t spf;     // sweeps_per_flat_check
  int active;       // 0 = free slot
};
struct BatchWalker {
  int slot;
  int W;
};
// What the host reads of a slot after a round: finished windows and the clocks.
struct SlotReport {
  int32_t n_done;     // -1 for a free slot
  int32_t active;
  uint64_t sweeps;    // clock[0]
  uint64_t rounds;    // clock[1]
  uint64_t attempts;  // clock[2]: WL trials of all walkers (counted by the batched rounds)
};

}  // namespace rewl
