/*
 * rewl.h -- C ABI of a GB300 (sm_103a) library for replica-exchange
 * Wang-Landau (REWL) sampling of 2D lattice spin models, after Vogel, Li,
 * Wuest, Landau, "A generic, hierarchical framework for massively parallel
 * Wang-Landau sampling", PRL 110, 210603 (2013).
 *
 * The method (paper, WL paragraph, Fig. 1, Eq. (1) and the paragraph after
 * it): the energy range is split into h overlapping windows; each window
 * holds m independent Wang-Landau walkers with their own ln g(E) and H(E);
 * walkers accept single-site moves with min[1, g(E_old)/g(E_new)], add
 * ln f to ln g and 1 to H at their energy after every trial; walkers of
 * neighbouring windows swap configurations with probability Eq. (1); when
 * every walker of a window has a flat H, the window's m ln g tables are
 * averaged and handed back, H is reset and ln f is halved; the run ends when
 * every window has reached ln f_final, and the fragments are joined where
 * d ln g / dE of neighbouring windows agree best.
 *
 * Conventions of every call:
 *  - every call returns a rewl_status; no exception crosses the ABI;
 *  - out-parameters are written only on REWL_OK;
 *  - all buffers passed in are HOST memory owned by the caller; the library
 *    owns all device memory of a handle (allocated with cudaMalloc, or with
 *    the caller's rewl_params.alloc hook) and frees it in rewl_destroy;
 *  - a handle is used by one host thread at a time;
 *  - inputs are copied at creation; the library keeps no caller pointer.
 *  - rewl_last_error() gives a one-line description of the last failure of
 *    the calling thread.
 */
#ifndef REWL_H
#define REWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rewl_ctx* rewl_handle;

typedef enum {
  REWL_OK = 0,
  REWL_EINVAL = 1,     /* invalid argument (see rewl_last_error) */
  REWL_ENOMEM = 2,     /* device or host allocation failed */
  REWL_ECUDA = 3,      /* a CUDA runtime call failed */
  REWL_ETIMEOUT = 4,   /* rewl_params.timeout_ms elapsed before done */
  REWL_EENTRY = 5,     /* a walker could not reach its energy window */
  REWL_EOVERFLOW = 6,  /* a histogram counter would overflow */
  REWL_EBUSY = 7,      /* server: no capacity (request stays queued) */
  REWL_ENOTFOUND = 8,  /* server: unknown request id */
  REWL_ENODEV = 9      /* no CUDA device, or the device is not sm_103 */
} rewl_status;

typedef enum { REWL_ISING = 0, REWL_POTTS = 1, REWL_EA_PM_J = 2, REWL_EA_PM_J_3D = 3 } rewl_model_kind;

/* Model: kind; q = number of Potts states (2..16), ignored otherwise.
 * Ising: E = -sum_<ij> s_i s_j; +-J: E = -sum_<ij> J_ij s_i s_j with
 * J_ij = +-1; Potts: E = -sum_<ij> delta(s_i, s_j).  The sum runs over the
 * 2N nearest-neighbour bonds of the periodic square lattice;
 * REWL_EA_PM_J_3D is the +-J glass on the periodic L x L x L cube (the
 * paper's 12^3 spin glass), 3N bonds, site i = (z L + y) L + x. */
typedef struct {
  int32_t kind;
  int32_t q;
} rewl_model;

/* Lattice: dim 2 with Lx == Ly == L, 2 <= L <= 256 (L even for +-J); or
 * dim 3 (REWL_EA_PM_J_3D only) with Lx == Ly == L the edge of the cube,
 * L even, 2 <= L <= 64; periodic must be 1. */
typedef struct {
  int32_t dim, Lx, Ly, periodic;
} rewl_lattice;

/* Optional device allocator (e.g. PyTorch's caching allocator): returns a
 * device pointer of at least `bytes` bytes usable on `stream`, or NULL. */
typedef void* (*rewl_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*rewl_free_fn)(void* ptr, void* stream, void* user);

enum { REWL_MODE_PLAIN = 0, REWL_MODE_GRAPH = 1 };

typedef struct {
  int32_t sweeps_per_exchange;   /* sweeps between exchange rounds; default 100 */
  int32_t sweeps_per_flat_check; /* sweeps between flatness checks; default 1000; a multiple of the above */
  double lnf0;                   /* initial ln f; default 1.0; must be a power of two */
  int32_t entry_max_sweeps;      /* budget of each greedy walk into a window; default 1000 */
  int32_t discovery_sweeps;      /* +-J only: zero-temperature descent fixing the energy range; default 200 */
  int64_t timeout_ms;            /* rewl_step returns REWL_ETIMEOUT after this wall time; 0 = none */
  void* stream;                  /* cudaStream_t to run on; NULL = a stream owned by the handle */
  int32_t lanes_per_walker;      /* G lanes cooperate on one walker (1,2,4,8,16,32); 0 = autotune */
  int32_t walkers_per_block;     /* walkers per CTA of the sweep kernel; 0 = autotune */
  int32_t mode;                  /* REWL_MODE_PLAIN: one launch per phase; REWL_MODE_GRAPH: the
                                    phases of one flatness period replayed as a captured CUDA graph */
  rewl_alloc_fn alloc;           /* NULL = cudaMalloc / cudaFree */
  rewl_free_fn free;
  void* alloc_user;
  int32_t profile;               /* 1 = time every sweep launch with CUDA events on the solve's stream
                                    (plain mode); read back through rewl_info */
  int32_t sweep_variant;         /* sweep kernel form, identical results: REWL_SWEEP_AUTO (default: the
                                    ring form when the solve has at most 8 walkers per SM and lanes / walkers
                                    per block are not forced, else the chain form), REWL_SWEEP_CHAIN
                                    (two-deep chain), REWL_SWEEP_STAGED (staged one-deep chain),
                                    REWL_SWEEP_RING (the chain with its draws made by a second, producer warp
                                    of the CTA; 32 lanes and one walker per CTA) */
  int32_t prefetch_draws;        /* 1 = in plain mode with variant 0 the draws of the next block (sites,
                                    ln u, conflict masks) are prepared on a second stream while the current
                                    block runs, when both buffers fit in 1 GiB; 0 = no (default: kernels
                                    running beside the sweep slow its chains) */
  int32_t wl_rule;               /* how ln f falls (the WL "update/convergence rule"): REWL_RULE_FLAT or
                                    REWL_RULE_ONE_OVER_T; see below */
  const int32_t* window_starts;  /* NULL: the equal partition of Fig. 1a from `windows` and `overlap`.
                                    Else `windows` first bins (global, 0-based) of an explicit partition,
                                    e.g. the run-time balanced one of Fig. 1b from rewl_plan_windows;
                                    read at rewl_create.  Must cover bins 0 .. n_bins-1 with widths >= 3,
                                    strictly increasing starts and ends, neighbours sharing >= 1 bin */
  const int32_t* window_widths;  /* `windows` widths in bins, with window_starts (both or neither) */
  int64_t wait_cycles;           /* bound of the ring form's hand-off waits between a walker's warp and
                                    its producer warp, in SM clock cycles from the start of a sweep
                                    launch; 0 = 2^34 (about 8 s at 2 GHz, while a launch takes
                                    milliseconds).  When a wait runs out both warps stop early and
                                    rewl_step returns REWL_ETIMEOUT at its next flatness check */
  int32_t server_walker_target;  /* served form: no request is admitted while at least this many walkers of
                                    windows not yet done are running (the first always is); 0 = 24 per SM,
                                    -1 = no such limit (slots and memory only) */
} rewl_params;

/*
 * WL rules.  REWL_RULE_FLAT: when every walker of a window is flat at a check
 * (min H * n >= flatness * sum H over its visited bins), the window merges and
 * ln f halves (f -> sqrt f; WL paragraph and the merge paragraph after
 * Eq. (1)).  REWL_RULE_ONE_OVER_T: the 1/t rule (Belardinelli and Pereyra,
 * PRE 75, 046701 (2007)), which the paper names as one the exchange works
 * with.  t = sweep_clock * N / window_bins (trials per energy level).  Stage
 * 0: at a check where every walker of the window has H > 0 on all its
 * visited bins, the window merges and halves ln f = 2^-k, unless
 * t < 2^(k+1) -- then it keeps ln f and enters stage 1.  Stage 1: at each
 * check with t >= 2^(k+1) the window merges and halves ln f, so ln f stays a
 * power of two with 1/t <= ln f < 2/t.  Both rules end a window when
 * ln f < lnf_final.
 */
enum { REWL_RULE_FLAT = 0, REWL_RULE_ONE_OVER_T = 1 };
enum { REWL_SWEEP_AUTO = -1, REWL_SWEEP_CHAIN = 0, REWL_SWEEP_STAGED = 1, REWL_SWEEP_RING = 2 };

/* Fills *p with the defaults above. */
void rewl_params_default(rewl_params* p);

/*
 * rewl_create -- set up one REWL solve on the current CUDA device.
 * Paper: windows and walkers (Fig. 1a caption and the paragraph after it),
 * the WL parameters (WL paragraph: f schedule ln f -> ln f/2, f_final).
 *
 *  out                 receives the handle (untouched on error)
 *  model, lattice      see above
 *  couplings           +-J only: 2N values +-1, site-major, [2*i] the bond
 *                      from site i = y*L + x to its right neighbour, [2*i+1] to
 *                      the one below; NULL = drawn with p = 1/2 from `seed`.
 *                      Must be NULL for Ising and Potts.
 *  windows             h >= 1 energy windows of equal width
 *  overlap             o in (0, 1): fraction of a window shared with the next
 *  walkers_per_window  m >= 1 independent walkers per window
 *  flatness            in (0, 1]: H is flat when min H >= flatness * mean H
 *                      over the bins the walker has visited (ln g > 0)
 *  lnf_final           > 0: a window is done when ln f < lnf_final
 *  seed                64-bit key of every Philox4x32-10 stream of the solve
 *  params              NULL = rewl_params_default
 *
 * Energy bins: Ising [-2N, 2N] step 4; Potts [-2N, 0] step 1; +-J step 4
 * over [E0, -E0], E0 the lowest energy a zero-temperature descent of all
 * walkers reaches (g(E) = g(-E) on the bipartite torus).  Windows: w =
 * ceil(B / (1 + (h-1)(1-o))) bins, window k starts at k(B-w)/(h-1) rounded
 * half up.  Each walker walks greedily into its window (REWL_EENTRY if it
 * cannot within the budget, also after a restart from the ground state or,
 * for +-J, from the lowest configuration found).
 * Errors: REWL_EINVAL (arguments), REWL_ENOMEM, REWL_ECUDA, REWL_ENODEV,
 * REWL_EENTRY.
 */
rewl_status rewl_create(rewl_handle* out, const rewl_model* model, const rewl_lattice* lattice,
                        const int8_t* couplings, int32_t windows, double overlap, int32_t walkers_per_window,
                        double flatness, double lnf_final, uint64_t seed, const rewl_params* params);

/*
 * rewl_step -- advance the solve.  Paper: WL walk (WL paragraph), exchange
 * (Eq. (1)), flatness / merge / f-reduction and termination (paragraph
 * after Eq. (1)).  Runs blocks of sweeps_per_exchange sweeps (one sweep =
 * N trial moves per walker), each followed by one exchange round and, every
 * sweeps_per_flat_check sweeps, by the flatness check, until at least
 * max_sweeps sweeps ran or every window is done.  max_sweeps <= 0 runs to
 * completion.  *done (may be NULL) = 1 when every window reached lnf_final.
 * Errors: REWL_EINVAL (NULL handle), REWL_ECUDA, REWL_ETIMEOUT (state stays
 * consistent; call again to continue), REWL_EOVERFLOW.
 */
rewl_status rewl_step(rewl_handle h, int64_t max_sweeps, int32_t* done);

/*
 * rewl_get_lng -- the joined, normalised ln g over the whole energy range
 * (paper, paragraph after Eq. (1): fragments are joined where the inverse
 * microcanonical temperatures d ln g/dE agree best).  Each window
 * contributes the mean of its walkers' ln g; window a+1 is shifted to match
 * window a at the overlap bin with the smallest difference of central
 * differences.  Normalised so that sum_E g(E) = 2^N (Ising, +-J) or q^N.
 *  lng       caller buffer of `capacity` doubles; bin b is energy
 *            e_min + b * e_step; bins never visited are -INFINITY
 *  n_bins, e_min, e_step  out (may be NULL)
 * Errors: REWL_EINVAL (capacity < number of bins, or no visited bin shared
 * by two neighbouring windows), REWL_ECUDA.
 */
rewl_status rewl_get_lng(rewl_handle h, double* lng, int32_t capacity, int32_t* n_bins, int32_t* e_min,
                         int32_t* e_step);

/*
 * rewl_get_window_lng -- raw ln g of one walker (walker in [0, m)) of one
 * window (or, with walker = -1, the mean over the window's walkers), w
 * values; local bin b is global bin bin_lo + b.  0 = never visited.
 * Errors: REWL_EINVAL (index or capacity), REWL_ECUDA.
 */
rewl_status rewl_get_window_lng(rewl_handle h, int32_t window, int32_t walker, double* lng, int32_t capacity,
                                int32_t* bin_lo, int32_t* n);

/* Sizes and counters of a solve. */
typedef struct {
  int32_t model, q, L, N;
  int32_t windows, walkers_per_window, window_bins, n_bins;
  int32_t e_min, e_max, e_step;
  int32_t lattice_words;     /* 32-bit words per walker configuration */
  int32_t lanes_per_walker, walkers_per_block, mode, windows_done;
  int64_t sweep_clock;       /* sweeps done by the solve (all active walkers) */
  int64_t exchange_rounds;
  int64_t attempts;          /* WL trial moves done by all walkers (entry walks excluded) */
  int64_t sweep_launches;    /* sweep-kernel launches timed (params.profile = 1) */
  double sweep_ms;           /* their summed device time, CUDA events on the solve's stream */
  int64_t h2d_bytes;         /* bytes copied host -> device by this handle so far */
  int64_t d2h_bytes;         /* bytes copied device -> host by this handle so far */
  int32_t prefetch_draws;    /* 1 when the next block's draws are prepared on a second stream */
  int32_t sweep_variant;     /* the sweep form in use (REWL_SWEEP_CHAIN, _STAGED or _RING) */
} rewl_info;

rewl_status rewl_get_info(rewl_handle h, rewl_info* info);

/*
 * Full state of a solve, for parity checks and checkpoint / resume.  Every
 * pointer is a caller-owned host buffer or NULL (skipped).  Walker W = a*m+k
 * is walker k of window a.
 *  lattice   [walkers][lattice_words] u32: Ising/+-J 1 bit per site, row y
 *            in words [y*Wr, (y+1)*Wr), Wr = ceil(L/32), site (x,y) = bit
 *            x%32 of word x/32 (bit 1 = spin -1); Potts 4 bits per site,
 *            Wr = ceil(L/8), site (x,y) = bits 4(x%8).. of word x/8
 *  E         [walkers] i32 current energy
 *  lng, H    [walkers][window_bins] f64 / u32, window-local bins
 *  win_start [windows] first global bin; lnf [windows]; iteration, done
 *  wl_accept, near_ties, exact_tests [walkers] u64: accepted WL moves;
 *            acceptance tests with |ln u - Delta ln g| < 1e-12; tests that
 *            needed the FP64 logarithm
 *  x_tried, x_accepted [windows] u64: exchange pairs of window pair (a,a+1)
 *  stage     [windows] i32: stage of the 1/t rule (REWL_RULE_ONE_OVER_T)
 */
typedef struct {
  uint32_t* lattice;
  int32_t* E;
  double* lng;
  uint32_t* H;
  int32_t* win_start;
  double* lnf;
  int32_t* iteration;
  int32_t* done;
  uint64_t* wl_accept;
  uint64_t* near_ties;
  uint64_t* exact_tests;
  uint64_t* x_tried;
  uint64_t* x_accepted;
  int64_t sweep_clock;
  int64_t exchange_rounds;
  int32_t* stage;       /* [windows] 1/t rule stage (0 or 1); optional, NULL reads as all 0 */
  int32_t* win_width;   /* [windows] bins of each window (read only; lng/H rows have window_bins =
                           the largest width, bins past a window's width stay 0) */
  int64_t* first_iter;  /* [windows] sweep clock at which the window's first merge happened, -1 before;
                           optional on set */
  int32_t* rep_id;      /* [walkers] the replica (configuration, followed through the exchanges) that
                           walker W holds; at creation walker W holds replica W */
  int32_t* rep_state;   /* [replicas] 0 = not yet in the lowest window, 1 = has been there, 2 = has since
                           reached the highest window */
  int64_t* rep_trips;   /* [replicas] completed round trips lowest -> highest -> lowest window (Fig. 3);
                           the three replica arrays are optional on set (all three or none) */
} rewl_state;

/* Copies the device state into the caller's buffers.  Errors: REWL_EINVAL,
 * REWL_ECUDA. */
rewl_status rewl_get_state(rewl_handle h, rewl_state* st);

/*
 * rewl_autotune -- picks the sweep kernel's launch shape for one problem by
 * timing candidates on the problem itself: the ring form (32 lanes and a
 * producer warp per walker) and the chain form with 32, 16, 8, 4 and 2 lanes
 * per walker (walkers per CTA as rewl_create chooses).  Each candidate is a
 * fresh rewl_create with the given arguments, one warm-up block, then `sweeps`
 * sweeps timed with CUDA events around every sweep launch.  All candidates
 * compute the same bits.  results: caller array of `capacity` entries, one per
 * candidate tried (*n_results); *best: `params` (or the defaults) with
 * sweep_variant, lanes_per_walker and walkers_per_block of the fastest, ready
 * for rewl_create.  Errors: REWL_EINVAL (arguments, sweeps not a multiple of
 * sweeps_per_exchange, no candidate ran); a candidate's own failure is in its
 * result's status.
 */
typedef struct {
  int32_t sweep_variant, lanes_per_walker, walkers_per_block;
  int32_t status;           /* rewl_status of the candidate's run */
  double ms_per_launch;     /* mean device time of one sweep launch (sweeps_per_exchange sweeps) */
  double attempts_per_s;    /* trials per second of sweep-kernel time */
} rewl_tune_result;

rewl_status rewl_autotune(const rewl_model* model, const rewl_lattice* lattice, const int8_t* couplings,
                          int32_t windows, double overlap, int32_t walkers_per_window, double flatness,
                          double lnf_final, uint64_t seed, const rewl_params* params, int32_t sweeps,
                          rewl_tune_result* results, int32_t capacity, int32_t* n_results, rewl_params* best);

/*
 * rewl_plan_windows -- the run-time balanced partition of Fig. 1b: windows
 * sized so that each finishes its first WL iteration after about the same
 * number of sweeps, estimated from a pre-run (the speed-up paragraph).  The
 * paper gives no formula; reading: a window's first iteration is a diffusive
 * walk lasting (sum over its bins of rho(b))^2; pre-run window a, which first
 * merged after first_iter_sweeps[a] sweeps (rewl_state.first_iter) and has
 * pre_widths[a] bins, gives rho_a = sqrt(first_iter_sweeps[a]) /
 * pre_widths[a]; rho(b) is the mean of rho_a over the pre-run windows holding
 * bin b.  The new `windows` windows are the equal partition of Fig. 1a with
 * overlap o laid out in the coordinate U(b) = rho(0) + ... + rho(b-1): each
 * carries the same sum of rho.  Host-only arithmetic (no device).  Output:
 * starts / widths, `windows` values each, for rewl_params.window_starts /
 * window_widths.  Errors: REWL_EINVAL (a pre-run window without a first
 * merge, a partition that would not pass rewl_create's checks).
 */
rewl_status rewl_plan_windows(const int64_t* first_iter_sweeps, const int32_t* pre_starts, const int32_t* pre_widths,
                              int32_t pre_windows, int32_t n_bins, int32_t windows, double overlap, int32_t* starts,
                              int32_t* widths);

/* Restores a state previously read from a handle created with the same
 * arguments (checkpoint / resume); lattice, E, lng, H, lnf, iteration, done
 * are required, counters optional.  Because every draw is a function of
 * (seed, walker, attempt index), a resumed run continues bit-identically.
 * Errors: REWL_EINVAL, REWL_ECUDA. */
rewl_status rewl_set_state(rewl_handle h, const rewl_state* st);

/* Frees all device and host memory of the handle.  NULL-safe. */
void rewl_destroy(rewl_handle h);

/*
 * rewl_thermo -- canonical thermodynamics from a density of states (the
 * paper's opening paragraph: WL gives the free energy at any temperature from
 * one simulation).  For each temperature T_i > 0 (k_B = 1, beta = 1/T) with
 * w(E) = g(E) exp(-beta E):
 *   out[5i+0] = ln Z = ln sum_E w(E)
 *   out[5i+1] = U = <E>
 *   out[5i+2] = C = beta^2 (<E^2> - <E>^2)   (centred two-pass sum)
 *   out[5i+3] = F = -T ln Z
 *   out[5i+4] = S = (U - F) / T
 * lng: n_bins values (host), bin b at energy e_min + b * e_step, -INFINITY for
 * levels that do not exist (e.g. rewl_get_lng's output); temperatures: n_T
 * values (host); out: 5 * n_T doubles (host).  All quantities are totals
 * (divide by N for per-site values).  FP64 throughout.
 * Errors: REWL_EINVAL (sizes, non-positive temperature, no finite ln g),
 * REWL_ENOMEM, REWL_ECUDA.
 */
rewl_status rewl_thermo(const double* lng, int32_t n_bins, int32_t e_min, int32_t e_step, const double* temperatures,
                        int32_t n_T, double* out);

/*
 * rewl_thermo_jackknife -- the quantities of rewl_thermo with statistical
 * errors by resampling over independent runs (the paper's join paragraph
 * determines errors by resampling; jackknife as in Newman and Barkema,
 * section 3.4.3).  lng_runs: n_runs >= 2 normalised ln g tables of one
 * problem, [n_runs][n_bins] row-major on the host (e.g. rewl_get_lng of runs
 * with different seeds); a bin counts only where every run is finite.
 * est[5i+q]: quantity q of the mean ln g over all runs at temperature i
 * (layout of rewl_thermo's out); err[5i+q] = sqrt((R-1)/R * sum_r (Q_(r) -
 * mean_r Q_(r))^2), Q_(r) from the mean without run r.  Host buffers of
 * 5 * n_T doubles.  Errors: REWL_EINVAL (sizes, temperatures, no bin finite in
 * every run), REWL_ENOMEM, REWL_ECUDA.
 */
rewl_status rewl_thermo_jackknife(const double* lng_runs, int32_t n_runs, int32_t n_bins, int32_t e_min,
                                  int32_t e_step, const double* temperatures, int32_t n_T, double* est, double* err);

/*
 * Served form.  The paper runs one solve at a time (one walker per CPU core,
 * conclusion paragraph); here many independent REWL solves -- different
 * models, lattice sizes, disorder realisations -- run together on one GPU.
 * Each request is exactly the method of rewl_create / rewl_step (WL
 * paragraph, Eq. (1), merge paragraph) with its own seed and schedule, so its
 * result is bit-identical to the one it gets alone.
 *
 * Requests are queued at submission (inputs are copied) and admitted first
 * come, first served while a slot (max_running), the device-memory budget
 * and the target of running walkers (rewl_params.server_walker_target: the
 * walkers of windows not yet done) allow; the memory a request may need is
 * estimated from its sizes with the widest window its energy range allows.
 * As windows finish, their walkers stop and make room for new requests.
 * Running requests are grouped by shape (model, L); a shape whose round of
 * sweeps_per_exchange sweeps lasts milliseconds gives each request a group of
 * its own (those rounds are latency-bound per walker; fused, every request
 * would wait for the slowest walker of all).  A group advances by
 * rounds: for every request of the group one block of sweeps_per_exchange
 * sweeps, one exchange round and, when due, the flatness check -- one fused
 * launch for the sweeps of all the group's walkers (with a producer warp per
 * walker while the GPU holds few walkers, else 4 walkers of a request per
 * CTA), one launch each for the exchanges, clocks and flatness checks of all
 * its requests.  Every phase boundary is decided on the device (clocks,
 * flatness, merges and done flags are device state; the kernels of finished
 * windows and requests do nothing), so a group's k rounds and the report read
 * after them are captured once as a CUDA graph and replayed, k adapted so
 * that a replay lasts a few milliseconds.  Each group runs on a stream of its
 * own, so groups of different sizes progress side by side at their own pace.
 * rewl_server_run issues a replay for every idle group and returns once at
 * least one has finished, per unit of max_rounds; it releases the server's
 * lock while it waits on the GPU.  Finished requests are retired when their
 * group's replay is read: their joined ln g is read back (rewl_server_result)
 * and their memory returns to the budget.  The server is internally
 * synchronised: any thread may call it.
 */
typedef struct rewl_server* rewl_server_handle;

typedef struct {
  rewl_model model;
  rewl_lattice lattice;
  const int8_t* couplings;       /* +-J only, as rewl_create; copied at submission */
  int32_t windows;
  double overlap;
  int32_t walkers_per_window;
  double flatness;
  double lnf_final;
  uint64_t seed;
} rewl_request;

enum { REWL_REQ_QUEUED = 0, REWL_REQ_RUNNING = 1, REWL_REQ_DONE = 2, REWL_REQ_FAILED = 3, REWL_REQ_CANCELLED = 4 };

typedef struct {
  int32_t state;        /* REWL_REQ_* */
  int32_t error;        /* rewl_status of a failed request */
  double queued_ms;     /* submission -> admission (or end, if never admitted) */
  double run_ms;        /* admission -> end */
  double latency_ms;    /* submission -> end (so far, if not ended) */
  int64_t sweeps;       /* sweeps run */
  int64_t attempts;     /* WL trials of its walkers */
  int64_t device_bytes; /* budget charged while running */
} rewl_request_info;

typedef struct {
  int32_t running, queued, finished, failed;
  int64_t rounds, attempts, device_bytes_in_use;
} rewl_server_stats;

/* device_bytes: memory budget for running requests; max_running: request slots;
 * params: sweeps_per_exchange, sweeps_per_flat_check, lnf0, entry and
 * discovery budgets and allocator of every request, server_walker_target
 * (NULL = defaults);
 * params.stream: NULL = one stream per shape group (groups overlap on the
 * device), else every group and request runs on that one stream (in order);
 * params.timeout_ms > 0: rewl_server_run fails with REWL_ETIMEOUT when no
 * round finishes within that time.  Errors: REWL_EINVAL, REWL_ENOMEM, REWL_ECUDA. */
rewl_status rewl_server_create(rewl_server_handle* out, int64_t device_bytes, int32_t max_running,
                               const rewl_params* params);
/* Queues a request; *id identifies it.  Errors: REWL_EINVAL (malformed),
 * REWL_ENOMEM (larger than the whole budget).  Errors found at admission
 * (e.g. REWL_EENTRY) end the request in REWL_REQ_FAILED. */
rewl_status rewl_server_submit(rewl_server_handle s, const rewl_request* r, uint64_t* id);
/* Admits what fits, issues a replay of rounds for every idle group and waits
 * (without holding the server's lock) until at least one has finished;
 * repeated up to max_rounds times (stops early when nothing runs).
 * stats->rounds counts the group rounds finished so far.
 * *stats (may be NULL) describes the server afterwards.
 * Errors: REWL_ECUDA, REWL_ETIMEOUT. */
rewl_status rewl_server_run(rewl_server_handle s, int32_t max_rounds, rewl_server_stats* stats);
/* State, timings and counters of a request.  Errors: REWL_ENOTFOUND. */
rewl_status rewl_server_poll(rewl_server_handle s, uint64_t id, rewl_request_info* info);
/* The joined, normalised ln g of a finished request (as rewl_get_lng).
 * Errors: REWL_ENOTFOUND, REWL_EBUSY (not finished), REWL_EINVAL (capacity). */
rewl_status rewl_server_result(rewl_server_handle s, uint64_t id, double* lng, int32_t capacity, int32_t* n_bins,
                               int32_t* e_min, int32_t* e_step);
/* Removes a queued request or stops a running one (its memory is freed at
 * once; other requests are unaffected).  Errors: REWL_ENOTFOUND. */
rewl_status rewl_server_cancel(rewl_server_handle s, uint64_t id);
/* Frees everything the server holds.  NULL-safe. */
void rewl_server_destroy(rewl_server_handle s);

/*
 * rewl_sweep_noalloc -- WL sweeps of walkers whose state the CALLER holds in
 * its own device memory, without any allocation by the library.  The paper
 * has no counterpart: this entry point exists for callers that cannot let a
 * library allocate device memory when they run a sweep (code inside an arena
 * or pool it does not control, a runtime whose allocator must not be
 * re-entered, a process that reserved all device memory up front).
 *
 * It runs the same sweep kernel as rewl_step, with the same trials and the
 * same bit-exact results, for d->sweeps sweeps starting at sweep index
 * d->first_sweep (trial t = first_sweep * N + i), and nothing else: no
 * exchange, no flatness check.  All pointers are DEVICE pointers owned by the
 * caller, in the layouts of rewl_state: lattice [walkers][lattice_words],
 * E [walkers], lng and H [walkers][window_bins] (updated in place);
 * win_start and lnf [windows] (read only); coupling_bits (+-J only, else
 * NULL): two bit planes [right|down][L][ceil(L/32)], bit set = J = -1.
 * stream: cudaStream_t or NULL (legacy stream); the call is asynchronous on it.
 *
 * Inputs the kernel checks on the device, per walker: E must lie in its
 * window (win_start[a] .. win_start[a] + window_bins - 1 in global bins) and
 * the window's lnf must be a power of two in [2^-39, 64].  A walker that
 * fails either is skipped (its state is left as it was) and its entry of
 * d->status, when given, is set to REWL_EINVAL; walkers that ran get 0.
 * d->status is an optional DEVICE array of [walkers] int32 owned by the
 * caller, written on the stream like the state; with NULL the statuses are
 * not reported.
 *
 * Working memory (walker list, internal status flags, sweep clock, counters)
 * comes from one fixed array of about 128 KB compiled into the library, room
 * for REWL_NOALLOC_MAX_WALKERS walkers; every GPU that loads the library
 * keeps it until the process exits.  Every call on a device uses the same
 * array and overwrites what the previous call left there (it clears what
 * must start at zero itself), so calls whose work overlaps on the GPU race:
 * order them on one stream or synchronise between them.  The first call on
 * each device looks up the array's device address and keeps it: make that
 * first call before any stream capture, and during set-up -- with CUDA's lazy
 * module loading it is also the call that loads the library's device code,
 * which the driver does with an allocation of its own.  The kept address
 * belongs to the device's primary context; after cudaDeviceReset on that
 * device the entry point must not be called again in the same process.
 * Errors: REWL_EINVAL (NULL pointer, bad descriptor, more than
 * REWL_NOALLOC_MAX_WALKERS walkers, window too wide for shared memory),
 * REWL_ENODEV, REWL_ECUDA.
 */
#define REWL_NOALLOC_MAX_WALKERS 4096
typedef struct {
  int32_t model, q, L;                        /* as rewl_create (dim 2, periodic; REWL_ISING, _POTTS, _EA_PM_J) */
  int32_t windows, walkers_per_window;        /* walker W = a * walkers_per_window + k */
  int32_t window_bins;                        /* w: bins of every window, and the row stride of lng and H */
  int32_t e_min, e_step;                      /* energy of global bin b = e_min + b * e_step */
  uint64_t seed;                              /* Philox key of the solve */
  uint64_t first_sweep;                       /* sweep index of the first sweep */
  int32_t sweeps;                             /* sweeps to run (>= 0) */
  int32_t lanes_per_walker;                   /* 1, 2, 4, 8, 16 or 32; 0 = 32 */
  int32_t* status;                            /* optional device [walkers]: 0 ran, REWL_EINVAL skipped */
} rewl_sweep_desc;

rewl_status rewl_sweep_noalloc(const rewl_sweep_desc* d, uint32_t* lattice, int32_t* E, double* lng, uint32_t* H,
                               const uint32_t* coupling_bits, const int32_t* win_start, const double* lnf,
                               void* stream);

/* Static description of a status code. */
const char* rewl_status_str(rewl_status s);

/* One-line description of the last failure in the calling thread. */
const char* rewl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* REWL_H */
