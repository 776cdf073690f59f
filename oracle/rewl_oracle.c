/*
 * rewl_oracle.c -- plain, single-threaded CPU oracle for replica-exchange
 * Wang-Landau (REWL) sampling of 2D lattice spin models.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this code.  It shares no
 * source, header, table or helper with the CUDA library; it implements the
 * method from the paper (Vogel, Li, Wuest, Landau, "A generic, hierarchical
 * framework for massively parallel Wang-Landau sampling", PRL 110, 210603):
 *
 *   - standard WL walk (paper, paragraph "The standard WL algorithm"):
 *     accept a trial move with P = min[1, g(E_old)/g(E_new)], then
 *     g(E) -> f g(E) and H(E) += 1 at the current energy;  when H is flat,
 *     reset H and reduce f (f -> sqrt f, i.e. ln f -> ln f / 2);
 *   - energy splitting into h overlapping windows (paper, Fig. 1a caption,
 *     and the paragraph after it), m independent walkers per window;
 *   - replica exchange between neighbouring windows with acceptance Eq. (1);
 *   - per-walker flatness, then averaging of the m estimators of one window
 *     and a simultaneous step to the next iteration (paragraph after Eq. (1));
 *   - termination when every window has reached f_final (same paragraph).
 *
 * Everything is written in the order the paper states it, with one FP64
 * operation per arithmetic step; no blocking, fusion or reordering.  Where
 * the paper is silent the reading used is stated at the point of use (entry
 * into windows, the exchange pairing, the "visited bins" flatness set, the
 * mean of ln g at merging, the random-number mapping).
 *
 * Spins are stored one per byte: 0/1 for Ising and +-J (s = 1 - 2b), 0..q-1
 * for Potts.  Site i = y*L + x on an L x L periodic square lattice.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "rewl_oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random       */
/* numbers: as easy as 1, 2, 3"): 10 rounds of the Philox S-box on a 128-bit */
/* counter with a 64-bit key bumped by the Weyl constants between rounds.   */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { /* key schedule: bump before every round but the first */
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream tags (4th counter word).  Every draw of the method has its own
 * (counter, key) so that any implementation can reproduce it. */
enum { TAG_FLIP = 0, TAG_ENTRY = 1, TAG_PERM = 2, TAG_XACC = 3, TAG_INIT = 4, TAG_COUPLING = 5 };

static void draw(const orc_rewl* R, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4] = {c0, c1, c2, tag};
  uint32_t key[2] = {(uint32_t)R->seed, (uint32_t)(R->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* floor(r * n / 2^32): an index in [0, n) from one 32-bit word. */
static uint32_t scale32(uint32_t r, uint32_t n) { return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32); }

/* Uniform u in (0,1) from two words: 52 random bits k, u = (2k+1) / 2^53
 * (exact in FP64, never 0 or 1). */
static double uniform_open01(uint32_t r2, uint32_t r3) {
  uint64_t k = ((uint64_t)r2 << 20) | (uint64_t)(r3 >> 12);
  return (double)(2 * k + 1) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* Model: energy and its change under a single-site move.                  */
/* ------------------------------------------------------------------------ */
/* Site i = (z L + y) L + x (z = 0 in 2D); neighbours on the periodic lattice. */
static int site_at(const orc_rewl* R, int x, int y, int z) { return (z * R->L + y) * R->L + x; }
static int right_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, (x + 1) % L, y, z); }
static int left_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, (x + L - 1) % L, y, z); }
static int down_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, x, (y + 1) % L, z); }
static int up_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, x, (y + L - 1) % L, z); }
static int back_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, x, y, (z + 1) % L); }
static int front_of(const orc_rewl* R, int i) { int L = R->L, x = i % L, y = (i / L) % L, z = i / (L * L); return site_at(R, x, y, (z + L - 1) % L); }

static int ising_s(uint8_t b) { return 1 - 2 * (int)b; }

/* Bond energy between sites i and j joined by coupling J (Ising / +-J):
 * -J s_i s_j.  Potts: -delta(s_i, s_j). */
static int bond_energy(const orc_rewl* R, int J, uint8_t a, uint8_t b) {
  if (R->model == ORC_POTTS) return -(a == b ? 1 : 0);
  return -J * ising_s(a) * ising_s(b);
}

/* Full energy E = sum over the dim N bonds (right, down and, in 3D, behind
 * every site). */
int orc_energy(const orc_rewl* R, const uint8_t* s) {
  int E = 0;
  for (int i = 0; i < R->N; ++i) {
    E += bond_energy(R, R->Jr[i], s[i], s[right_of(R, i)]);
    E += bond_energy(R, R->Jd[i], s[i], s[down_of(R, i)]);
    if (R->dim == 3) E += bond_energy(R, R->Jb[i], s[i], s[back_of(R, i)]);
  }
  return E;
}

/* Energy change when site i takes value v_new: the 2 dim bonds at i. */
static int delta_energy(const orc_rewl* R, const uint8_t* s, int i, uint8_t v_new) {
  int r = right_of(R, i), l = left_of(R, i), d = down_of(R, i), u = up_of(R, i);
  int before = bond_energy(R, R->Jr[i], s[i], s[r]) + bond_energy(R, R->Jr[l], s[l], s[i]) +
               bond_energy(R, R->Jd[i], s[i], s[d]) + bond_energy(R, R->Jd[u], s[u], s[i]);
  int after = bond_energy(R, R->Jr[i], v_new, s[r]) + bond_energy(R, R->Jr[l], s[l], v_new) +
              bond_energy(R, R->Jd[i], v_new, s[d]) + bond_energy(R, R->Jd[u], s[u], v_new);
  if (R->dim == 3) {
    int b = back_of(R, i), f = front_of(R, i);
    before += bond_energy(R, R->Jb[i], s[i], s[b]) + bond_energy(R, R->Jb[f], s[f], s[i]);
    after += bond_energy(R, R->Jb[i], v_new, s[b]) + bond_energy(R, R->Jb[f], s[f], v_new);
  }
  return after - before;
}

/* The proposal of one single-site move from the 4 words of one draw:
 * site from r0; Potts: a new value uniform over the q-1 other values
 * (symmetric proposal, so the WL acceptance is unchanged); Ising/+-J: flip. */
static void propose(const orc_rewl* R, const uint8_t* s, const uint32_t r[4], int* site, uint8_t* v_new) {
  *site = (int)scale32(r[0], (uint32_t)R->N);
  if (R->model == ORC_POTTS)
    *v_new = (uint8_t)((s[*site] + 1 + scale32(r[1], (uint32_t)(R->q - 1))) % (uint32_t)R->q);
  else
    *v_new = (uint8_t)(1 - s[*site]);
}

/* ------------------------------------------------------------------------ */
/* Energy bins and the window partition (paper, Fig. 1a: equal-size windows */
/* with overlap o).                                                         */
/* ------------------------------------------------------------------------ */
static int bin_of(const orc_rewl* R, int E) { return (E - R->e_min) / R->e_step; }

/* Window width w = ceil(B / (1 + (h-1)(1-o))) bins; starts are k(B-w)/(h-1)
 * rounded half up, so the first window starts at bin 0 and the last ends at
 * bin B-1.  (The paper gives no rounding rule; this is the reading used.)
 * A partition given explicitly (Fig. 1b: run-time balanced windows of
 * unequal width) must start at bin 0, end at bin B-1, have widths >= 3,
 * strictly increasing starts and ends, and neighbours sharing >= 1 bin. */
static int make_windows(orc_rewl* R, int core_lo, int core_bins) {
  int B = R->n_bins, h = R->h;
  if (R->params.window_starts) {
    const int32_t* st = R->params.window_starts;
    const int32_t* wd = R->params.window_widths;
    if (!wd || st[0] != 0 || st[h - 1] + wd[h - 1] != B) return ORC_EINVAL;
    R->w = 0;
    for (int k = 0; k < h; ++k) {
      if (wd[k] < 3 || st[k] < 0 || st[k] + wd[k] > B) return ORC_EINVAL;
      if (k > 0 && (st[k] <= st[k - 1] || st[k] + wd[k] <= st[k - 1] + wd[k - 1] || st[k] > st[k - 1] + wd[k - 1] - 1))
        return ORC_EINVAL;
      R->win_start[k] = st[k];
      R->win_width[k] = wd[k];
      if (wd[k] > R->w) R->w = wd[k];
    }
    return ORC_OK;
  }
  if (h == 1) {
    R->w = B;
    R->win_start[0] = 0;
    R->win_width[0] = B;
    return ORC_OK;
  }
  /* the equal partition of the core [core_lo, core_lo + core_bins); the first
   * and the last window then reach down to bin 0 and up to bin B-1 */
  int Bc = core_bins;
  double wd = ceil((double)Bc / (1.0 + (double)(h - 1) * (1.0 - R->overlap)));
  int w = (int)wd;
  if (w > Bc) w = Bc;
  if (w < 3) return ORC_EINVAL;
  for (int k = 0; k < h; ++k) {
    int64_t num = 2 * (int64_t)k * (int64_t)(Bc - w) + (h - 1);
    R->win_start[k] = core_lo + (int)(num / (2 * (int64_t)(h - 1)));
    R->win_width[k] = w;
  }
  for (int k = 0; k + 1 < h; ++k)
    if (R->win_start[k + 1] > R->win_start[k] + w - 1) return ORC_EINVAL; /* neighbours must overlap */
  R->win_width[0] += R->win_start[0];
  R->win_start[0] = 0;
  R->win_width[h - 1] = B - R->win_start[h - 1];
  R->w = 0;
  for (int k = 0; k < h; ++k)
    if (R->win_width[k] > R->w) R->w = R->win_width[k];
  return ORC_OK;
}

static int win_lo_E(const orc_rewl* R, int a) { return R->e_min + R->win_start[a] * R->e_step; }
static int win_hi_E(const orc_rewl* R, int a) { return R->e_min + (R->win_start[a] + R->win_width[a] - 1) * R->e_step; }
static int in_window(const orc_rewl* R, int a, int E) { return E >= win_lo_E(R, a) && E <= win_hi_E(R, a); }

/* ------------------------------------------------------------------------ */
/* Accessors                                                                */
/* ------------------------------------------------------------------------ */
static uint8_t* spins_of(orc_rewl* R, int W) { return R->spins + (size_t)W * R->N; }
static double* lng_of(orc_rewl* R, int W) { return R->lng + (size_t)W * R->w; }
static uint32_t* H_of(orc_rewl* R, int W) { return R->H + (size_t)W * R->w; }

/* ------------------------------------------------------------------------ */
/* Initial state and entry into the windows (the paper is silent on how a   */
/* walker reaches its window; the reading used: a greedy walk that accepts  */
/* a move iff it does not increase the distance to the window, with a       */
/* deterministic restart from a known low-energy configuration).            */
/* ------------------------------------------------------------------------ */
static void init_lattice(orc_rewl* R, int W) {
  uint8_t* s = spins_of(R, W);
  uint32_t r[4];
  if (R->model == ORC_POTTS) {
    for (int i = 0; i < R->N; ++i) {
      if (i % 4 == 0) draw(R, (uint32_t)(i / 4), 0, (uint32_t)W, TAG_INIT, r);
      s[i] = (uint8_t)scale32(r[i % 4], (uint32_t)R->q);
    }
  } else {
    for (int i = 0; i < R->N; ++i) {
      if (i % 128 == 0) draw(R, (uint32_t)(i / 128), 0, (uint32_t)W, TAG_INIT, r);
      s[i] = (uint8_t)((r[(i % 128) / 32] >> (i % 32)) & 1u);
    }
  }
}

static int distance_to_window(const orc_rewl* R, int a, int E) {
  if (E < win_lo_E(R, a)) return win_lo_E(R, a) - E;
  if (E > win_hi_E(R, a)) return E - win_hi_E(R, a);
  return 0;
}

/* One greedy move on the entry stream of walker W: accept iff the
 * objective (distance to the window, or E itself while searching for low
 * energies) does not increase. */
static void greedy_move(orc_rewl* R, int W, int target_window) {
  uint8_t* s = spins_of(R, W);
  uint32_t r[4];
  uint64_t t = R->entry_t[W]++;
  draw(R, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, TAG_ENTRY, r);
  int site;
  uint8_t v_new;
  propose(R, s, r, &site, &v_new);
  int E_new = R->E[W] + delta_energy(R, s, site, v_new);
  int before = target_window < 0 ? R->E[W] : distance_to_window(R, target_window, R->E[W]);
  int after = target_window < 0 ? E_new : distance_to_window(R, target_window, E_new);
  if (after <= before) {
    s[site] = v_new;
    R->E[W] = E_new;
  }
}

static int enter_window(orc_rewl* R, int W, int a) {
  int64_t budget = (int64_t)R->params.entry_max_sweeps * R->N;
  for (int64_t n = 0; n < budget && distance_to_window(R, a, R->E[W]) > 0; ++n) greedy_move(R, W, a);
  if (distance_to_window(R, a, R->E[W]) == 0) return ORC_OK;
  /* restart from the reference low-energy configuration */
  memcpy(spins_of(R, W), R->seed_config, (size_t)R->N);
  R->E[W] = orc_energy(R, spins_of(R, W));
  for (int64_t n = 0; n < budget && distance_to_window(R, a, R->E[W]) > 0; ++n) greedy_move(R, W, a);
  return distance_to_window(R, a, R->E[W]) == 0 ? ORC_OK : ORC_EENTRY;
}

/* ------------------------------------------------------------------------ */
/* Creation                                                                 */
/* ------------------------------------------------------------------------ */
void orc_default_params(orc_params* p) {
  p->sweeps_per_exchange = 100;
  p->sweeps_per_flat_check = 1000;
  p->lnf0 = 1.0;
  p->entry_max_sweeps = 1000;
  p->discovery_sweeps = 200;
  p->wl_rule = 0;
}

int orc_create(orc_rewl** out, int model, int q, int L, const int8_t* couplings, int h, double overlap, int m,
               double flatness, double lnf_final, uint64_t seed, const orc_params* params) {
  *out = NULL;
  orc_params P;
  if (params) P = *params; else orc_default_params(&P);
  if (model < 0 || model > 3 || L < 2 || L > 256 || h < 1 || m < 1 || h * m > (1 << 20)) return ORC_EINVAL;
  if (model == ORC_POTTS && (q < 2 || q > 16)) return ORC_EINVAL;
  if ((model == ORC_EA || model == ORC_EA3) && (L % 2) != 0) return ORC_EINVAL;
  if (model == ORC_EA3 && L > 64) return ORC_EINVAL;
  if (!(overlap > 0.0 && overlap < 1.0) || !(flatness > 0.0 && flatness <= 1.0) || !(lnf_final > 0.0)) return ORC_EINVAL;
  if (!(P.lnf0 >= lnf_final) || P.sweeps_per_exchange < 1 || P.sweeps_per_flat_check < P.sweeps_per_exchange ||
      P.sweeps_per_flat_check % P.sweeps_per_exchange != 0 || P.entry_max_sweeps < 1 || P.discovery_sweeps < 0 ||
      (P.wl_rule != 0 && P.wl_rule != 1))
    return ORC_EINVAL;
  if (model != ORC_EA && model != ORC_EA3 && couplings != NULL) return ORC_EINVAL;

  orc_rewl* R = (orc_rewl*)calloc(1, sizeof(orc_rewl));
  R->model = model; R->q = (model == ORC_POTTS) ? q : 2; R->L = L;
  R->dim = model == ORC_EA3 ? 3 : 2;
  R->N = R->dim == 3 ? L * L * L : L * L;
  R->h = h; R->m = m; R->overlap = overlap; R->flatness = flatness; R->lnf_final = lnf_final; R->seed = seed;
  R->params = P;
  int N = R->N, n_walkers = h * m;
  R->Jr = (int8_t*)malloc((size_t)N);
  R->Jd = (int8_t*)malloc((size_t)N);
  R->Jb = (int8_t*)malloc((size_t)N);
  /* couplings: Ising and Potts J = 1; +-J either given (dim N values: right,
   * down and, in 3D, behind of every site) or drawn with p = 1/2 from the
   * request seed (bond b = dim i + d is bit b of the coupling stream). */
  int n_negative = 0, D = R->dim;
  for (int i = 0; i < N; ++i) {
    int j[3] = {1, 1, 1};
    if (model == ORC_EA || model == ORC_EA3) {
      for (int d = 0; d < D; ++d) {
        if (couplings) {
          j[d] = couplings[D * i + d];
          if (j[d] != 1 && j[d] != -1) { orc_destroy(R); return ORC_EINVAL; }
        } else {
          uint32_t r[4];
          int b = D * i + d;
          draw(R, (uint32_t)(b / 128), 0, 0xFFFFFFFFu, TAG_COUPLING, r);
          j[d] = ((r[(b % 128) / 32] >> (b % 32)) & 1u) ? -1 : 1;
        }
      }
    }
    R->Jr[i] = (int8_t)j[0];
    R->Jd[i] = (int8_t)j[1];
    R->Jb[i] = (int8_t)j[2];
    n_negative += (j[0] < 0) + (j[1] < 0) + (D == 3 && j[2] < 0);
  }
  R->spins = (uint8_t*)calloc((size_t)n_walkers * N, 1);
  R->E = (int*)calloc((size_t)n_walkers, sizeof(int));
  R->entry_t = (uint64_t*)calloc((size_t)n_walkers, sizeof(uint64_t));
  R->seed_config = (uint8_t*)calloc((size_t)N, 1);
  R->win_start = (int*)calloc((size_t)h, sizeof(int));
  R->win_width = (int*)calloc((size_t)h, sizeof(int));
  R->first_iter = (int64_t*)malloc((size_t)h * sizeof(int64_t));
  for (int a = 0; a < h; ++a) R->first_iter[a] = -1;
  R->lnf = (double*)calloc((size_t)h, sizeof(double));
  R->iter = (int*)calloc((size_t)h, sizeof(int));
  R->done = (int*)calloc((size_t)h, sizeof(int));
  R->phase = (int*)calloc((size_t)h, sizeof(int));
  R->wl_accept = (uint64_t*)calloc((size_t)n_walkers, sizeof(uint64_t));
  R->near_ties = (uint64_t*)calloc((size_t)n_walkers, sizeof(uint64_t));
  R->x_tried = (uint64_t*)calloc((size_t)h, sizeof(uint64_t));
  R->x_accepted = (uint64_t*)calloc((size_t)h, sizeof(uint64_t));
  R->rep_id = (int32_t*)calloc((size_t)n_walkers, sizeof(int32_t));
  R->rep_state = (int32_t*)calloc((size_t)n_walkers, sizeof(int32_t));
  R->rep_trips = (int64_t*)calloc((size_t)n_walkers, sizeof(int64_t));
  for (int W = 0; W < n_walkers; ++W) {
    R->rep_id[W] = W;
    R->rep_state[W] = W < m ? 1 : 0; /* the replicas that start in the lowest window */
  }

  for (int W = 0; W < n_walkers; ++W) {
    init_lattice(R, W);
    R->E[W] = orc_energy(R, spins_of(R, W));
  }

  /* Energy range.  Ising: [-2N, 2N] in steps of 4.  Potts: [-2N, 0] in
   * steps of 1.  +-J (2D and 3D): steps of 4 with E = -dim N + 2 n_neg
   * (mod 4).  A zero-temperature descent of every walker finds E_d (the
   * lowest energy any walker reaches); the windows are laid out over the
   * core [E_d, -E_d] (g(E) = g(-E) on the bipartite periodic lattice: flip
   * one sublattice), and the lowest and highest windows reach on to the
   * bounds of the grid, e_min = E_d - 4 floor((E_d + dim N) / 4) >= -dim N and
   * e_max = -e_min, so the walk can still find energies below E_d (no energy
   * is locked out; bins never visited stay out of the flatness test). */
  int core_lo = 0, core_bins = 0;
  if (model == ORC_ISING) {
    R->e_min = -2 * N; R->e_max = 2 * N; R->e_step = 4;
  } else if (model == ORC_POTTS) {
    R->e_min = -2 * N; R->e_max = 0; R->e_step = 1;
  } else {
    R->e_step = 4;
    int64_t descent = (int64_t)P.discovery_sweeps * N;
    int best = 0x7fffffff, best_W = 0;
    for (int W = 0; W < n_walkers; ++W) {
      for (int64_t n = 0; n < descent; ++n) greedy_move(R, W, -1);
      if (R->E[W] < best) { best = R->E[W]; best_W = W; }
    }
    (void)n_negative;
    if (best >= 0) { orc_destroy(R); return ORC_EENTRY; }
    core_lo = (best + R->dim * N) / 4;
    R->e_min = best - 4 * core_lo; R->e_max = -R->e_min;
    core_bins = (-2 * best) / 4 + 1;
    memcpy(R->seed_config, spins_of(R, best_W), (size_t)N);
  }
  R->n_bins = (R->e_max - R->e_min) / R->e_step + 1;
  if (core_bins == 0) core_bins = R->n_bins;
  if (make_windows(R, core_lo, core_bins) != ORC_OK) { orc_destroy(R); return ORC_EINVAL; }
  /* Ising / Potts restart configuration: the ground state (all b = 0). */
  if (model != ORC_EA && model != ORC_EA3) memset(R->seed_config, 0, (size_t)N);

  R->lng = (double*)calloc((size_t)n_walkers * R->w, sizeof(double));
  R->H = (uint32_t*)calloc((size_t)n_walkers * R->w, sizeof(uint32_t));
  for (int a = 0; a < h; ++a) R->lnf[a] = P.lnf0;

  for (int W = 0; W < n_walkers; ++W) {
    int st = enter_window(R, W, W / m);
    if (st != ORC_OK) { orc_destroy(R); return st; }
  }
  *out = R;
  return ORC_OK;
}

void orc_destroy(orc_rewl* R) {
  if (!R) return;
  free(R->Jr); free(R->Jd); free(R->Jb); free(R->spins); free(R->E); free(R->entry_t); free(R->seed_config);
  free(R->win_start); free(R->win_width); free(R->first_iter); free(R->lnf); free(R->iter); free(R->done); free(R->phase); free(R->lng); free(R->H);
  free(R->wl_accept); free(R->near_ties); free(R->x_tried); free(R->x_accepted);
  free(R->rep_id); free(R->rep_state); free(R->rep_trips);
  free(R);
}

/* ------------------------------------------------------------------------ */
/* One WL trial move of walker W at attempt index t (paper, "The standard   */
/* WL algorithm": P = min[1, g(E_old)/g(E_new)], then g(E) -> f g(E) and    */
/* H(E) += 1 at the energy the walker is at after the move).                */
/* ------------------------------------------------------------------------ */
static void wl_attempt(orc_rewl* R, int W, uint64_t t) {
  int a = W / R->m;
  uint8_t* s = spins_of(R, W);
  double* lng = lng_of(R, W);
  uint32_t* H = H_of(R, W);
  uint32_t r[4];
  draw(R, (uint32_t)t, (uint32_t)(t >> 32), (uint32_t)W, TAG_FLIP, r);
  int site;
  uint8_t v_new;
  propose(R, s, r, &site, &v_new);
  int E_old = R->E[W];
  int E_new = E_old + delta_energy(R, s, site, v_new);
  int accept = 0;
  if (in_window(R, a, E_new)) { /* moves that leave the window are rejected */
    int b_old = bin_of(R, E_old) - R->win_start[a];
    int b_new = bin_of(R, E_new) - R->win_start[a];
    double delta = lng[b_old] - lng[b_new];           /* ln[g(E_old)/g(E_new)] */
    if (delta >= 0.0) {
      accept = 1;                                      /* min[1, ratio] = 1 */
    } else {
      double u = uniform_open01(r[2], r[3]);
      double lu = log(u);
      if (fabs(lu - delta) < 1e-12) R->near_ties[W]++;
      accept = lu < delta;                             /* u < g(E_old)/g(E_new) */
    }
  }
  if (accept) {
    s[site] = v_new;
    R->E[W] = E_new;
    R->wl_accept[W]++;
  }
  int b = bin_of(R, R->E[W]) - R->win_start[a];
  lng[b] = lng[b] + R->lnf[a];                         /* ln g(E) += ln f */
  H[b] = H[b] + 1u;                                    /* H(E) += 1 */
}

/* ------------------------------------------------------------------------ */
/* Replica exchange between windows a and a+1 (paper, Eq. (1)).  The paper  */
/* says walker i picks a partner j in a neighbouring window at random; the  */
/* reading used: in exchange round r the window pairs (a, a+1) with         */
/* a = r (mod 2) are active, and walker k of window a is paired with walker */
/* sigma(k) of window a+1, sigma a uniform random permutation (Fisher-Yates).*/
/* Windows that are done are frozen and take no part.                       */
/* ------------------------------------------------------------------------ */
static void exchange_pair(orc_rewl* R, int a, uint32_t round) {
  int m = R->m;
  int* sigma = (int*)malloc((size_t)m * sizeof(int));
  for (int k = 0; k < m; ++k) sigma[k] = k;
  for (int i = m - 1; i >= 1; --i) {
    uint32_t r[4];
    draw(R, round, (uint32_t)a, (uint32_t)i, TAG_PERM, r);
    int j = (int)scale32(r[0], (uint32_t)(i + 1));
    int tmp = sigma[i]; sigma[i] = sigma[j]; sigma[j] = tmp;
  }
  for (int k = 0; k < m; ++k) {
    int Wi = a * m + k;                 /* walker i in window a, holds X */
    int Wj = (a + 1) * m + sigma[k];    /* walker j in window a+1, holds Y */
    int EX = R->E[Wi], EY = R->E[Wj];
    R->x_tried[a]++;
    if (!in_window(R, a + 1, EX) || !in_window(R, a, EY)) continue;
    double* gi = lng_of(R, Wi);
    double* gj = lng_of(R, Wj);
    int iX = bin_of(R, EX) - R->win_start[a], iY = bin_of(R, EY) - R->win_start[a];
    int jX = bin_of(R, EX) - R->win_start[a + 1], jY = bin_of(R, EY) - R->win_start[a + 1];
    /* ln P = [ln g_i(E(X)) - ln g_i(E(Y))] + [ln g_j(E(Y)) - ln g_j(E(X))] */
    double d1 = gi[iX] - gi[iY];
    double d2 = gj[jY] - gj[jX];
    double D = d1 + d2;
    int accept;
    if (D >= 0.0) {
      accept = 1;
    } else {
      uint32_t r[4];
      draw(R, round, (uint32_t)a, (uint32_t)k, TAG_XACC, r);
      double lu = log(uniform_open01(r[2], r[3]));
      if (fabs(lu - D) < 1e-12) R->near_ties[Wi]++;
      accept = lu < D;
    }
    if (accept) {
      /* swap configurations X <-> Y; the ln g and H stay with the walkers */
      uint8_t* si = spins_of(R, Wi);
      uint8_t* sj = spins_of(R, Wj);
      for (int n = 0; n < R->N; ++n) { uint8_t t = si[n]; si[n] = sj[n]; sj[n] = t; }
      R->E[Wi] = EY;
      R->E[Wj] = EX;
      R->x_accepted[a]++;
      /* the replicas travel with their configurations (Fig. 3: round trips) */
      int32_t ri = R->rep_id[Wj], rj = R->rep_id[Wi];
      R->rep_id[Wi] = ri;
      R->rep_id[Wj] = rj;
      if (a == 0) { /* replica ri arrives in the lowest window */
        if (R->rep_state[ri] == 2) R->rep_trips[ri]++;
        R->rep_state[ri] = 1;
      }
      if (a + 1 == R->h - 1 && R->rep_state[rj] == 1) R->rep_state[rj] = 2; /* rj reaches the highest */
    }
  }
  free(sigma);
}

/* ------------------------------------------------------------------------ */
/* Flatness and merging (paper, paragraph after Eq. (1)): every walker must */
/* be flat on its own; when all m walkers of a window are flat at the same  */
/* check, their estimators are averaged and handed back to all of them, H   */
/* is reset and ln f is halved (f -> sqrt f).  "Flat" is not defined in the */
/* paper; the reading used: over the bins the walker has visited (ln g > 0),*/
/* min H >= flatness * mean H.  The average is the mean of ln g.            */
/* ------------------------------------------------------------------------ */
int orc_walker_is_flat(const orc_rewl* R, int W) {
  const double* lng = R->lng + (size_t)W * R->w;
  const uint32_t* H = R->H + (size_t)W * R->w;
  uint64_t S = 0;
  uint32_t hmin = 0xffffffffu;
  int n = 0;
  for (int b = 0; b < R->win_width[W / R->m]; ++b) {
    if (lng[b] > 0.0) {
      ++n;
      S += H[b];
      if (H[b] < hmin) hmin = H[b];
    }
  }
  if (n == 0) return 0;
  return (double)hmin * (double)n >= R->flatness * (double)S;
}

/* The m estimators of window a are averaged (mean of ln g, summed in walker */
/* order) and handed back to all of them; H is reset.                        */
static void merge_window(orc_rewl* R, int a) {
  int m = R->m;
  if (R->iter[a] == 0) R->first_iter[a] = (int64_t)R->sweep_clock; /* end of the first iteration */
  for (int b = 0; b < R->win_width[a]; ++b) {
    double sum = lng_of(R, a * m)[b];
    for (int k = 1; k < m; ++k) sum = sum + lng_of(R, a * m + k)[b];
    double mean = sum / (double)m;
    for (int k = 0; k < m; ++k) {
      lng_of(R, a * m + k)[b] = mean;
      H_of(R, a * m + k)[b] = 0u;
    }
  }
  R->iter[a] += 1;
}

static void halve_lnf(orc_rewl* R, int a) {
  R->lnf[a] = R->lnf[a] * 0.5; /* f -> sqrt(f) */
  if (R->lnf[a] < R->lnf_final) R->done[a] = 1; /* this window reached f_final */
}

static void flatness_and_merge(orc_rewl* R, int a) {
  int m = R->m;
  for (int k = 0; k < m; ++k)
    if (!orc_walker_is_flat(R, a * m + k)) return;
  merge_window(R, a);
  halve_lnf(R, a);
}

/* ------------------------------------------------------------------------ */
/* The 1/t rule (Belardinelli and Pereyra, PRE 75, 046701 (2007)), which    */
/* the paper names as one of the WL rules replica exchange works with.  In  */
/* its first stage ln f is halved whenever every energy has been visited    */
/* again (H(E) > 0 everywhere); once a halving would take ln f below 1/t,   */
/* ln f follows 1/t, where t is the Monte Carlo time in trials per energy   */
/* level.  Reading used here (the paper gives no details):                  */
/*   - t of window a = (trials per walker) / w_a = sweep_clock * N / w_a;   */
/*   - stage 0 test at each check: every walker of the window has H > 0 in  */
/*     every bin it has visited (ln g > 0); then the window merges and      */
/*     either halves ln f = 2^-k, or, when 2^-(k+1) < 1/t (i.e.             */
/*     sweep_clock*N < w*2^(k+1)), keeps ln f and enters stage 1;           */
/*   - stage 1: ln f stays a power of two and follows 1/t from above: at a  */
/*     check where t >= 2^(k+1) the window merges and halves ln f, so       */
/*     1/t <= ln f < 2/t at every check (one halving per check at most);    */
/*   - termination as in the flatness rule: ln f < ln f_final.              */
/* Keeping ln f a power of two keeps every ln g exact (merge paragraph).    */
/* ------------------------------------------------------------------------ */
int orc_walker_all_seen(const orc_rewl* R, int W) {
  const double* lng = R->lng + (size_t)W * R->w;
  const uint32_t* H = R->H + (size_t)W * R->w;
  int n = 0;
  for (int b = 0; b < R->win_width[W / R->m]; ++b) {
    if (lng[b] > 0.0) {
      ++n;
      if (H[b] == 0u) return 0;
    }
  }
  return n > 0;
}

static void one_over_t_step(orc_rewl* R, int a) {
  int m = R->m;
  int e2;
  frexp(R->lnf[a], &e2);               /* ln f = 0.5 * 2^e2 = 2^-k */
  int k = 1 - e2;
  uint64_t trials = R->sweep_clock * (uint64_t)R->N;
  /* w * 2^(k+1): t >= 2^(k+1) iff trials >= next (beyond 2^47 trials per level: never) */
  uint64_t next = k + 1 < 48 ? (uint64_t)R->win_width[a] << (k + 1) : UINT64_MAX;
  if (R->phase[a] == 0) {
    for (int j = 0; j < m; ++j)
      if (!orc_walker_all_seen(R, a * m + j)) return;
    merge_window(R, a);
    if (trials < next) R->phase[a] = 1; /* 2^-(k+1) < 1/t: follow 1/t from here */
    else halve_lnf(R, a);
  } else if (trials >= next) {
    merge_window(R, a);
    halve_lnf(R, a);
  }
}

/* ------------------------------------------------------------------------ */
/* The phase schedule: blocks of sweeps_per_exchange sweeps, then one       */
/* exchange round, then (every sweeps_per_flat_check sweeps) the flatness   */
/* check.  One sweep = N trial moves per walker.  Attempt t of a walker is  */
/* t = sweep_clock * N + i; all walkers of active windows move in lockstep. */
/* ------------------------------------------------------------------------ */
/* Number of windows not done yet. */
int orc_active_windows(const orc_rewl* R) {
  int active = 0;
  for (int a = 0; a < R->h; ++a) active += !R->done[a];
  return active;
}

/* The WL sweeps of the current block for walkers W0 .. W1-1 of the windows
 * not done.  A walker's sweeps read and write only its own configuration,
 * energy, ln g, H and counters, so disjoint walker ranges of one block may
 * run on different host threads (same trials, same results). */
void orc_block_sweeps(orc_rewl* R, int W0, int W1) {
  uint64_t t0 = R->sweep_clock * (uint64_t)R->N;
  uint64_t n_att = (uint64_t)R->params.sweeps_per_exchange * (uint64_t)R->N;
  for (int W = W0; W < W1 && W < R->h * R->m; ++W) {
    if (R->done[W / R->m]) continue;
    for (uint64_t i = 0; i < n_att; ++i) wl_attempt(R, W, t0 + i);
  }
}

/* The rest of the block, after every walker's sweeps: the clock, one
 * exchange round and, when due, the flatness check of every window. */
void orc_block_finish(orc_rewl* R) {
  int h = R->h;
  R->sweep_clock += (uint64_t)R->params.sweeps_per_exchange;
  for (int a = (int)(R->xround % 2u); a + 1 < h; a += 2)
    if (!R->done[a] && !R->done[a + 1]) exchange_pair(R, a, R->xround);
  R->xround += 1u;
  if (R->sweep_clock % (uint64_t)R->params.sweeps_per_flat_check == 0)
    for (int a = 0; a < h; ++a) {
      if (R->done[a]) continue;
      if (R->params.wl_rule == 1) one_over_t_step(R, a);
      else flatness_and_merge(R, a);
    }
}

int orc_run_blocks(orc_rewl* R, int64_t n_blocks, int* all_done) {
  for (int64_t blk = 0; blk < n_blocks; ++blk) {
    if (!orc_active_windows(R)) break;
    orc_block_sweeps(R, 0, R->h * R->m);
    orc_block_finish(R);
  }
  if (all_done) *all_done = orc_active_windows(R) == 0;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors for tests                                                      */
/* ------------------------------------------------------------------------ */
void orc_info(const orc_rewl* R, int64_t* info) {
  info[0] = R->model; info[1] = R->q; info[2] = R->L; info[3] = R->N;
  info[4] = R->h; info[5] = R->m; info[6] = R->w; info[7] = R->n_bins;
  info[8] = R->e_min; info[9] = R->e_max; info[10] = R->e_step;
  info[11] = (int64_t)R->sweep_clock; info[12] = R->xround;
}

void orc_get_windows(const orc_rewl* R, int32_t* start, double* lnf, int32_t* iter, int32_t* done) {
  for (int a = 0; a < R->h; ++a) {
    if (start) start[a] = R->win_start[a];
    if (lnf) lnf[a] = R->lnf[a];
    if (iter) iter[a] = R->iter[a];
    if (done) done[a] = R->done[a];
  }
}

void orc_get_replicas(const orc_rewl* R, int32_t* rep_id, int32_t* rep_state, int64_t* rep_trips) {
  for (int W = 0; W < R->h * R->m; ++W) {
    if (rep_id) rep_id[W] = R->rep_id[W];
    if (rep_state) rep_state[W] = R->rep_state[W];
    if (rep_trips) rep_trips[W] = R->rep_trips[W];
  }
}

void orc_get_window_layout(const orc_rewl* R, int32_t* width, int64_t* first_iter) {
  for (int a = 0; a < R->h; ++a) {
    if (width) width[a] = R->win_width[a];
    if (first_iter) first_iter[a] = R->first_iter[a];
  }
}

void orc_get_phase(const orc_rewl* R, int32_t* phase) {
  for (int a = 0; a < R->h; ++a) phase[a] = R->phase[a];
}

void orc_get_walkers(const orc_rewl* R, uint8_t* spins, int32_t* E, double* lng, uint32_t* H) {
  size_t n = (size_t)R->h * R->m;
  if (spins) memcpy(spins, R->spins, n * R->N);
  if (E) for (size_t W = 0; W < n; ++W) E[W] = R->E[W];
  if (lng) memcpy(lng, R->lng, n * R->w * sizeof(double));
  if (H) memcpy(H, R->H, n * R->w * sizeof(uint32_t));
}

void orc_get_couplings(const orc_rewl* R, int8_t* J) {
  for (int i = 0; i < R->N; ++i) {
    J[R->dim * i] = R->Jr[i];
    J[R->dim * i + 1] = R->Jd[i];
    if (R->dim == 3) J[3 * i + 2] = R->Jb[i];
  }
}

void orc_get_counters(const orc_rewl* R, uint64_t* wl_accept, uint64_t* near_ties, uint64_t* x_tried,
                      uint64_t* x_accepted) {
  size_t n = (size_t)R->h * R->m;
  if (wl_accept) memcpy(wl_accept, R->wl_accept, n * sizeof(uint64_t));
  if (near_ties) memcpy(near_ties, R->near_ties, n * sizeof(uint64_t));
  if (x_tried) memcpy(x_tried, R->x_tried, (size_t)R->h * sizeof(uint64_t));
  if (x_accepted) memcpy(x_accepted, R->x_accepted, (size_t)R->h * sizeof(uint64_t));
}

/* Test hooks: overwrite a walker's ln g table or a window's ln f (used by the
 * detailed-balance test of Eq. (1), which freezes ln g with ln f = 0). */
void orc_set_walker_lng(orc_rewl* R, int W, const double* lng) { memcpy(lng_of(R, W), lng, (size_t)R->w * sizeof(double)); }
void orc_set_window_lnf(orc_rewl* R, int a, double lnf) { R->lnf[a] = lnf; }
void orc_set_walker_H(orc_rewl* R, int W, const uint32_t* H) { memcpy(H_of(R, W), H, (size_t)R->w * sizeof(uint32_t)); }
