/*
 * rewl_oracle.h -- interface of the plain CPU oracle for replica-exchange
 * Wang-Landau sampling.  TEST INFRASTRUCTURE ONLY: used by tests/,
 * __graft_entry__.smoke() and bench.py's CPU baseline; never by the library.
 */
#ifndef REWL_ORACLE_H
#define REWL_ORACLE_H
#include <stdint.h>

enum { ORC_ISING = 0, ORC_POTTS = 1, ORC_EA = 2, ORC_EA3 = 3 };  /* ORC_EA3: +-J on the L x L x L cube */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EENTRY = 5 };

typedef struct {
  int sweeps_per_exchange;    /* sweeps between exchange rounds (100) */
  int sweeps_per_flat_check;  /* sweeps between flatness checks (1000), a multiple of the above */
  double lnf0;                /* initial ln f (1.0) */
  int entry_max_sweeps;       /* budget of each greedy entry walk (1000 sweeps) */
  int discovery_sweeps;       /* +-J only: zero-temperature descent that fixes the energy range (200) */
  int wl_rule;                /* 0: flatness rule (f -> sqrt f on flat H); 1: the 1/t rule */
  const int32_t* window_starts; /* h first bins, or NULL for the equal partition (Fig. 1a) */
  const int32_t* window_widths; /* h widths in bins (with window_starts) */
} orc_params;

typedef struct orc_rewl {
  int model, q, L, N;
  int dim;                    /* 2, or 3 for ORC_EA3 (N = L^3, site i = (z L + y) L + x) */
  int8_t *Jr, *Jd, *Jb;       /* couplings of the bond to the right / below / behind (3D) each site */
  int e_min, e_max, e_step, n_bins;
  int h, m, w;
  double overlap, flatness, lnf_final;
  uint64_t seed;
  orc_params params;
  int* win_start;             /* first global bin of each window */
  int* win_width;             /* bins of each window (w is the largest) */
  int64_t* first_iter;        /* sweep clock of each window's first merge, -1 before it */
  double* lnf;
  int *iter, *done;
  int* phase;                 /* 1/t rule: 0 while ln f is halved on the histogram test, 1 once it follows 1/t */
  uint8_t* spins;             /* [h*m][N] */
  int* E;                     /* [h*m] */
  double* lng;                /* [h*m][w] */
  uint32_t* H;                /* [h*m][w] */
  uint8_t* seed_config;       /* restart configuration for the entry walk */
  uint64_t* entry_t;          /* per-walker counter of the entry stream */
  uint64_t sweep_clock;
  uint32_t xround;
  uint64_t *wl_accept, *near_ties, *x_tried, *x_accepted;
  /* replica round trips (Fig. 3): rep_id[W] = the configuration (replica) walker W
   * holds; per replica: rep_state 0 = not yet in the lowest window, 1 = has been
   * there (heading up), 2 = has since reached the highest window (heading down);
   * rep_trips = completed lowest -> highest -> lowest trips */
  int32_t *rep_id, *rep_state;
  int64_t* rep_trips;
} orc_rewl;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_default_params(orc_params* p);
int orc_create(orc_rewl** out, int model, int q, int L, const int8_t* couplings, int h, double overlap, int m,
               double flatness, double lnf_final, uint64_t seed, const orc_params* params);
void orc_destroy(orc_rewl* R);
int orc_run_blocks(orc_rewl* R, int64_t n_blocks, int* all_done);
int orc_active_windows(const orc_rewl* R);
void orc_block_sweeps(orc_rewl* R, int W0, int W1);
void orc_block_finish(orc_rewl* R);
int orc_energy(const orc_rewl* R, const uint8_t* s);
int orc_walker_is_flat(const orc_rewl* R, int W);
void orc_info(const orc_rewl* R, int64_t* info);
void orc_get_windows(const orc_rewl* R, int32_t* start, double* lnf, int32_t* iter, int32_t* done);
void orc_get_phase(const orc_rewl* R, int32_t* phase);
void orc_get_window_layout(const orc_rewl* R, int32_t* width, int64_t* first_iter);
void orc_get_replicas(const orc_rewl* R, int32_t* rep_id, int32_t* rep_state, int64_t* rep_trips);
int orc_walker_all_seen(const orc_rewl* R, int W);
void orc_get_walkers(const orc_rewl* R, uint8_t* spins, int32_t* E, double* lng, uint32_t* H);
void orc_get_couplings(const orc_rewl* R, int8_t* J);
void orc_get_counters(const orc_rewl* R, uint64_t* wl_accept, uint64_t* near_ties, uint64_t* x_tried,
                      uint64_t* x_accepted);
void orc_set_walker_lng(orc_rewl* R, int W, const double* lng);
void orc_set_window_lnf(orc_rewl* R, int a, double lnf);
void orc_set_walker_H(orc_rewl* R, int W, const uint32_t* H);

#endif
