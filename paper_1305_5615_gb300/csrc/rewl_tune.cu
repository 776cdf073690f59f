// rewl_tune.cu -- rewl_autotune: picks the sweep kernel's launch shape (form,
// lanes per walker, walkers per CTA) for one problem by timing candidates on
// the problem itself.  Every candidate computes the same bits (the sweep forms
// are bit-identical), so the choice changes speed only.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rewl.h"
#include "rewl_ctx.h"
#include "rewl_kernels.h"
#include "rewl_layout.h"

using namespace rewl;

namespace {

struct Candidate {
  int32_t variant, lanes, wpb;
};

}  // namespace

extern "C" rewl_status rewl_autotune(const rewl_model* model, const rewl_lattice* lattice, const int8_t* couplings,
                                     int32_t windows, double overlap, int32_t walkers_per_window, double flatness,
                                     double lnf_final, uint64_t seed, const rewl_params* params, int32_t sweeps,
                                     rewl_tune_result* results, int32_t capacity, int32_t* n_results,
                                     rewl_params* best) {
  if (!model || !lattice || !results || capacity < 1 || !n_results || !best || sweeps < 1) {
    rewl_set_last_error("rewl_autotune: invalid argument");
    return REWL_EINVAL;
  }
  rewl_params base;
  if (params) base = *params;
  else rewl_params_default(&base);
  if (sweeps % base.sweeps_per_exchange != 0) {
    rewl_set_last_error("rewl_autotune: sweeps must be a multiple of sweeps_per_exchange");
    return REWL_EINVAL;
  }
  // candidates: the ring form (one walker per CTA with a producer warp), and the chain form
  // with 32, 16, 8, 4 and 2 lanes per walker, walkers per CTA chosen by rewl_create
  std::vector<Candidate> cand = {{REWL_SWEEP_RING, 32, 1}, {REWL_SWEEP_CHAIN, 32, 0}, {REWL_SWEEP_CHAIN, 16, 0},
                                 {REWL_SWEEP_CHAIN, 8, 0}, {REWL_SWEEP_CHAIN, 4, 0}, {REWL_SWEEP_CHAIN, 2, 0}};
  int n = 0, best_i = -1;
  double best_ms = 0.0;
  for (const Candidate& cd : cand) {
    if (n >= capacity) break;
    rewl_params p = base;
    p.sweep_variant = cd.variant;
    p.lanes_per_walker = cd.lanes;
    p.walkers_per_block = cd.wpb;
    p.mode = REWL_MODE_PLAIN;
    p.profile = 1;
    p.prefetch_draws = 0;
    rewl_tune_result& r = results[n];
    std::memset(&r, 0, sizeof r);
    r.sweep_variant = cd.variant;
    r.lanes_per_walker = cd.lanes;
    rewl_handle h = nullptr;
    rewl_status st = rewl_create(&h, model, lattice, couplings, windows, overlap, walkers_per_window, flatness,
                                 lnf_final, seed, &p);
    if (st == REWL_OK) st = rewl_step(h, base.sweeps_per_exchange, nullptr);  // warm-up block
    rewl_info i0{}, i1{};
    if (st == REWL_OK) st = rewl_get_info(h, &i0);
    if (st == REWL_OK) st = rewl_step(h, sweeps, nullptr);
    if (st == REWL_OK) st = rewl_get_info(h, &i1);
    if (h) rewl_destroy(h);
    r.status = st;
    if (st == REWL_OK && i1.sweep_launches > i0.sweep_launches) {
      r.walkers_per_block = i1.walkers_per_block;
      r.sweep_variant = i1.sweep_variant;
      r.ms_per_launch = (i1.sweep_ms - i0.sweep_ms) / (double)(i1.sweep_launches - i0.sweep_launches);
      r.attempts_per_s = (double)(i1.attempts - i0.attempts) / ((i1.sweep_ms - i0.sweep_ms) * 1e-3);
      if (best_i < 0 || r.ms_per_launch < best_ms) {
        best_i = n;
        best_ms = r.ms_per_launch;
      }
    }
    ++n;
  }
  *n_results = n;
  if (best_i < 0) {
    rewl_set_last_error("rewl_autotune: no candidate ran");
    return REWL_EINVAL;
  }
  *best = base;
  best->sweep_variant = results[best_i].sweep_variant;
  best->lanes_per_walker = results[best_i].lanes_per_walker;
  best->walkers_per_block = results[best_i].walkers_per_block;
  return REWL_OK;
}
