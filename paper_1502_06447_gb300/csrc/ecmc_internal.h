// Internal declarations shared by the library's translation units.
#pragma once
#include <math.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/ecmc.h"

namespace ecmc {

// Device status codes (first failure wins).  DEV_BOUNDS (bounds-checked
// builds only, -DECMC_CHECKED): an index out of range was caught and the
// access skipped; the status word then holds DEV_BOUNDS | site << 8.
enum : int { DEV_OK = 0, DEV_STUCK = 1, DEV_CAPACITY = 2, DEV_TILE = 3, DEV_BOUNDS = 4 };

// Accumulator slots in the device counter array.
enum : int {
  CNT_EVENTS = ECMC_NEV,
  CNT_SWAP_TRIED = ECMC_NEV + 1,
  CNT_ECS = ECMC_NEV + 2,
  CNT_CONFIRMED = ECMC_NEV + 3,
  CNT_EXHAUSTIVE = ECMC_NEV + 4,
  CNT_N = ECMC_NEV + 5
};
enum : int { SUM_LIFT = 0, SUM_REFL = 1, SUM_DISP = 2, SUM_N = 3 };

// Host-side fault injection for tests: with ECMC_ALLOC_LIMIT=<bytes> in the
// environment, every device allocation of the library above that size
// fails as cudaMalloc does when the device is out of memory (the call then
// returns ECMC_ENOMEM); unset or 0: no limit.
inline bool alloc_refused(size_t bytes) {
  const char *e = getenv("ECMC_ALLOC_LIMIT");
  if (!e || !*e) return false;
  const unsigned long long lim = strtoull(e, nullptr, 10);
  return lim > 0 && bytes > lim;
}

// x > 0 rounded up to FP32 (host side)
inline float round_up_f32(double x) {
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
}

// One replica of a batch (device table): its box, tiles, cell grids, chain
// length, where its beads, cells and tiles start in the concatenated arrays,
// and its Philox key word.
struct RepParams {
  double L[3], half[3], T[3], W[3], cs[3];
  int32_t D[3], nc[3], lg[3];
  float linv[3], lorg;
  int32_t N;
  int32_t pad;
  int64_t bead_off;   // first bead in the concatenated position array
  int64_t cell_off;   // first cell in the concatenated cell arrays
  int64_t unit_off;   // first tile in the concatenated tile numbering
  int64_t n_beads;
  uint64_t replica;   // Philox key word 1
};

// Everything one EC launch needs, by value.
struct ECParams {
  // system
  int64_t n;
  int32_t N;
  double L[3], half[3];
  double sigma, sig2, b2;
  double s_cap;
  // decomposition (domain mode)
  int32_t domain;
  int32_t D[3];
  double T[3], W[3];
  double halo_hs, halo_te;
  int32_t nc[3];
  double cs[3];
  // run
  uint64_t seed, replica;
  int64_t sweep;        // domain: sweep index; serial: first EC ordinal
  int32_t ecs_per_tile; // domain: ECs per tile; serial: ECs in this launch
  double ell;
  int64_t event_cap;
  double p_swap;
  int32_t swap_mode;    // 0: never propose, 1: always, 2: draw u < p_swap
  uint64_t swap_thr;    // u53(w) < p_swap  <=>  (w >> 11) < swap_thr = ceil(p_swap 2^53)
  int32_t dir_mode;
  int32_t stage_cap;
  int32_t m_cap;        // motile slots with FP64 in shared memory (screened domain form)
  int32_t n_units;      // tiles (domain) or 1 (serial)
  // FP32 screen margins (units of sigma, sigma^2)
  float eps_v, eps_d, eps_x;
  float s_cap_f;  // s_cap rounded up to FP32 (the screen's cap on a free flight)
  // buffers
  double *r;
  int32_t *img;
  const double *cr;        // positions in cell order
  const int32_t *cid;      // ids in cell order
  const int32_t *ctag;     // tiles in cell order
  const int32_t *cstart;   // cell starts (ncell + 1)
  const float *crf;        // FP32 positions in cell order
  const float *rf;         // FP32 positions by bead
  unsigned long long *counters;
  double *sums;
  int *status;
  // per-EC records (may be null)
  uint64_t *rec_digest;
  double *rec_lift;
  int64_t *rec_events;
  int64_t rec_offset;
  int64_t rec_cap;
  ecmc_event *log;
  unsigned long long *log_n;
  int64_t log_cap;
  // batch: replica table (units are the concatenated tiles of all replicas),
  // the sweep counter on the device (graph replays advance it), and the
  // largest local grid over the replicas
  const RepParams *reps;
  int32_t n_reps;
  int32_t ncl_max;
  const int64_t *sweep_dev;
  int64_t rec_sweep0;
  // local cell grid of a tile (domain mode)
  int32_t lg[3];
  float linv[3];
  float lorg;
  // block-lockstep kernel: tiles per block (0: occupancy choice) and the
  // device counter its persistent blocks take units from (reset per launch)
  int32_t block_tiles;
  int32_t *unit_next;
  // slow push-off (plain FP64 domain kernel): the ECs of a tile start at its
  // flagged motile beads, one each in id order, and a pivot ignores the
  // beads it overlaps; null otherwise
  const uint8_t *po_flag;
  // push-off run from the device: the launch does nothing when no bead
  // overlaps (the count of the flag pass before it); null otherwise
  const unsigned long long *po_count;
  int32_t rq_per_tile;  // request list entries per tile of the block (1..6)
  // block-lockstep kernel: tight capacities for a first pass (0: none); a
  // tile that does not fit them is listed in `deferred` and run by a second
  // pass with stage_cap / m_cap (tiles are independent, so the events are
  // the same).  defer_mode: 0 one pass, 1 first pass, 2 second pass.
  int32_t stage_tight, m_tight;
  int32_t defer_mode;
  int32_t *deferred;
  int32_t *n_deferred;
  // bead-spring chains (Sec. II): k > 0 replaces every tether by a harmonic
  // spring (k/2)(b - sigma)^2; bond partners of motile beads are then staged
  // wherever they are (a spring has no longest bond)
  double k_spring;
};

// message for ecmc_last_error (ecmc_api.cu)
void set_last_error(const char *msg);

// launchers (k_ec.cu)
cudaError_t launch_ec(const ECParams &P, int lanes, int fp32f, cudaStream_t s);
cudaError_t launch_ec_batch(const ECParams &P, int lanes, int fp32f, cudaStream_t s);
size_t ec_smem_bytes(int stage_cap, int motile_cap, int ncell, int groups_per_block);
// block-lockstep kernel of the screened domain form (lanes 4, 8, 16)
cudaError_t launch_ec_lock(const ECParams &P, int lanes, cudaStream_t s);
cudaError_t launch_ec_lock_batch(const ECParams &P, int lanes, cudaStream_t s);
size_t lock_smem_bytes(int stage_cap, int motile_cap, int ncell, int tiles_per_block);

// cell list and domain tags (k_cells.cu)
struct CellParams {
  int64_t n;
  double L[3];
  int32_t nc[3];
  double cs[3];
  int32_t domain;
  int32_t D[3];
  double T[3], W[3];
  uint64_t seed, replica;
  int64_t sweep;
  const double *r;
  int32_t *tag;
  int32_t *cell;
  int32_t *rank;
  int32_t *count;     // ncell (zeroed by the launcher)
  int32_t *start;     // ncell + 1
  int32_t *block_sums;
  double *cr;
  int32_t *cid;
  int32_t *ctag;
  float *crf;         // FP32 positions in cell order (staging's halo test)
  float *rf;          // FP32 positions by bead (staging's shadows)
  const int64_t *sweep_dev;  // sweep index on the device (null: `sweep`)
  // bead-spring chains (domain mode): a bead whose bonded bead is motile in
  // another tile is immotile for the sweep, decided on the tags of k_tag_count
  // (`tag`); the final tags go to ctag and, by bead, to `ftag` (may be null)
  int32_t N;
  int32_t spring;
  int32_t *ftag;
};
cudaError_t launch_cells(const CellParams &C, int64_t ncell, cudaStream_t s);

// the same for a batch: all replicas' beads at once (per-bead replica index,
// replica table), concatenated cell grids, one counting sort
struct CellBatch {
  int64_t n;                 // beads over all replicas
  const double *r;
  const int32_t *rep_of;     // replica of each bead
  const RepParams *reps;
  uint64_t seed;
  const int64_t *sweep_dev;  // sweep counter on the device
  int32_t *tag;
  int32_t *cell;
  int32_t *rank;
  int32_t *count;
  int32_t *start;
  int32_t *block_sums;
  double *cr;
  int32_t *cid;              // id within the replica
  int32_t *ctag;
  float *crf;                // FP32 positions in cell order
  float *rf;                 // FP32 positions by bead (concatenated)
};
cudaError_t launch_cells_batch(const CellBatch &C, int64_t ncell_total, cudaStream_t s);
cudaError_t launch_sweep_advance(int64_t *sweep_dev, cudaStream_t s);
size_t cells_scratch_ints(int64_t ncell);

// observables (k_obs.cu)
struct ObsParams {
  int64_t n;
  int32_t N;
  double L[3], half[3];
  double sig2, b2;
  const double *r;
  const int32_t *img;
  const double *g1ref;     // 3 per chain or null
  // cell list over the current positions (for the overlap count)
  int32_t nc[3];
  const double *cr;
  const int32_t *cid;
  const int32_t *cstart;
  const int32_t *cell;     // cell of each bead
  double *out_d;           // [re2_sum, bond_max, bond_min, g1_sum, bond_sum]
  // [overlaps, tether_violations, contact pairs (2 shells), taut bonds (2 shells)]
  unsigned long long *out_u;
  // squared shell bounds: pairs [lo, s1), [s1, s2); bonds (t1, t0], (t2, t1]
  double c_lo, c_s1, c_s2, c_t0, c_t1, c_t2;
};
cudaError_t launch_obs(const ObsParams &O, cudaStream_t s);
// positions copied in as given: wrap into [0, L), fold boxes into img
cudaError_t launch_wrap(double *r, int32_t *img, int64_t n, const double L[3],
                        unsigned long long *bad, cudaStream_t s);
cudaError_t launch_g1_snapshot(const ObsParams &O, double *g1ref, cudaStream_t s);

// g1 table (Sec. IV, Eq. 3): middle-bead snapshots at K levels, level k
// taken every P^k sweeps into a ring of P slots, and the sums of squared
// displacements for the lags j P^k (j = 1 .. P-1) over chains and origins
struct G1Track {
  int64_t n;
  int32_t N;
  double L[3];
  const double *r;
  const int32_t *img;
  double *ring;              // [K][P][n / N][3]
  double *sum;               // [K][P - 1]
  unsigned long long *cnt;   // [K][P - 1]
  int32_t P, K;
  int64_t Pk[16];            // P^k
  int64_t t;                 // sweeps since tracking began (0: first snapshot)
};
cudaError_t launch_g1_track(const G1Track &G, cudaStream_t s);
// beads overlapping another at |d|^2 < thr (cell list of O), as 0/1 flags
cudaError_t launch_po_flags(const ObsParams &O, double thr, uint8_t *flag,
                            unsigned long long *count, cudaStream_t s);
// push-off sweep done on the device: when the flag pass counted overlaps,
// the sweep index and the sweeps run (ctr[0], ctr[1]) advance
cudaError_t launch_po_advance(const unsigned long long *count, int64_t *ctr, cudaStream_t s);
// phantom chains, unwrapped (k_obs.cu); bad counts walks that ran out of attempts
cudaError_t launch_phantom(int64_t nch, int N, const double L[3], double bond, double ct,
                           uint64_t seed, double *r, unsigned long long *bad, cudaStream_t s);

// Chain structure pass (k_struct.cu): per-chain record columns
// T = Tr S, lam1, lam2, lam3, b, c, kappa2, 4 b^2 + 3 c^2, g2 summand, |R_e|^2,
// then the middle bead relative to the centre of mass (3); the first
// STRUCT_SUMS columns are summed over chains in chain order.
enum : int { STRUCT_REC = 13, STRUCT_SUMS = 10 };
struct StructParams {
  int64_t n;
  int32_t N;
  double L[3], half[3];
  const double *r;
  double *u;                 // [n][3] positions along each chain
  double *rec;               // [n / N][STRUCT_REC]
  const double *mref;        // [n / N][3] g2 reference or null
  double *part;              // [n / N][N] R^2(n) partial sums (with r2n)
  double *r2n;               // [N] or null
  double *sums;              // [STRUCT_SUMS]
  unsigned long long *hist;  // [nbins] or null
  int64_t nbins;
  double dR;
};
cudaError_t launch_struct(const StructParams &S, cudaStream_t s);
cudaError_t launch_lattice(const int32_t dims[3], double a, double jitter,
                           uint64_t seed, uint64_t replica, double *r, int64_t n,
                           cudaStream_t s);

// Staging capacity for a box of sides E[3] (a tile plus its halo, or the
// motile part of a tile) at bead number density rho: the larger of a 30 %
// density-fluctuation margin, 1.3 rho V + 32, and the most sites a simple-
// cubic lattice of this density (spacing a = rho^(-1/3), jitter below
// 0.01 a) can put in the box, prod(floor((E_a + 0.02) / a) + 1) + 8: the
// lattice start is the densest arrangement these melts meet, and a box
// aligned with its planes holds floor(E/a) + 1 sites per axis.  Rounded up
// to a multiple of 32.
inline int32_t stage_bound(const double E[3], double rho) {
  const double a_inv = cbrt(rho);
  const double fluct = 1.3 * rho * E[0] * E[1] * E[2] + 32.0;
  double lat = 1.0;
  for (int a = 0; a < 3; ++a) lat *= floor((E[a] + 0.02) * a_inv) + 1.0;
  lat += 8.0;
  const double b = fluct > lat ? fluct : lat;
  const int64_t n = (int64_t)ceil(b);
  return (int32_t)((n + 31) / 32 * 32);
}

// Tight capacities of the block-lockstep kernel's first pass: `factor`
// times the mean occupancy of a melted tile plus a margin, rounded to 8
// (tiles that exceed them, e.g. at the lattice start, run in the second
// pass; a smaller factor fits more tiles per SM and defers more of them).
inline void tight_caps(const double E[3], const double Wm[3], double rho, int32_t full_stage,
                       int32_t full_m, int32_t *stage_t, int32_t *m_t, double factor = 1.08) {
  const double vs = E[0] * E[1] * E[2], vm = Wm[0] * Wm[1] * Wm[2];
  int64_t st = (int64_t)ceil(factor * rho * vs + 16.0);
  int64_t mt = (int64_t)ceil(1.2 * rho * vm + 12.0);
  st = (st + 7) / 8 * 8;
  mt = (mt + 7) / 8 * 8;
  *stage_t = (int32_t)(st < full_stage ? st : full_stage);
  *m_t = (int32_t)(mt < full_m ? mt : full_m);
  if (*m_t > *stage_t) *m_t = *stage_t;
}

// ---------------------------------------------------------------- autotuner
// One launch setting of the domain sweep.  The search is a coordinate
// descent: lanes per EC, tile side, global cell side, ECs per tile, and the
// staging of the block-lockstep kernel (warps per block, the first pass's
// capacity factor), each axis scanned with the others held at their best so
// far, in up to two rounds.  The
// objective is ECs per device-second (each EC displaces by ell, so this is
// the rate of progress of the Markov chain; events/s would reward small
// tiles for their extra wall reflections).
struct TunePoint {
  int lanes;
  double tile_side;  // in units of sigma
  double cell_side;  // in units of sigma
  int ecs;
  int warps;         // block lockstep: warps per block (tiles = warps 32 / lanes)
  double tight;      // block lockstep: first-pass capacity factor
};

struct TuneScore {
  double ecs_per_s = 0.0, events_per_s = 0.0;
};

// trial(point, &score) -> ECMC_OK (scored), ECMC_EINVAL (point not
// admissible for this system: skipped) or another status (abort).
template <class Trial>
ecmc_status tune_search(TunePoint start, Trial trial, TunePoint *best, TuneScore *best_score,
                        int *n_trials) {
  static const int lanes_c[] = {4, 8, 16, 32};
  static const double tile_c[] = {3.4, 3.8, 4.2, 4.6, 5.0, 6.0, 7.0};
  static const double cell_c[] = {1.05, 1.4};
  static const int ecs_c[] = {1, 2, 4, 8};
  static const int warps_c[] = {1, 2, 4};
  static const double tight_c[] = {1.0, 1.08, 1.16};
  TunePoint cur = start;
  TuneScore cur_s{};
  bool have = false;
  int n = 0;
  // points already timed (a second round revisits none of them)
  constexpr int VMAX = 128;
  TunePoint seen[VMAX];
  int nseen = 0;
  auto consider = [&](const TunePoint &pt) -> ecmc_status {
    for (int i = 0; i < nseen; ++i)
      if (seen[i].lanes == pt.lanes && seen[i].tile_side == pt.tile_side &&
          seen[i].cell_side == pt.cell_side && seen[i].ecs == pt.ecs && seen[i].warps == pt.warps &&
          seen[i].tight == pt.tight)
        return ECMC_OK;
    if (nseen < VMAX) seen[nseen++] = pt;
    TuneScore sc{};
    const ecmc_status st = trial(pt, &sc);
    if (st == ECMC_EINVAL) return ECMC_OK;
    if (st != ECMC_OK) return st;
    ++n;
    if (!have || sc.ecs_per_s > cur_s.ecs_per_s) {
      cur = pt;
      cur_s = sc;
      have = true;
    }
    return ECMC_OK;
  };
  ecmc_status st = consider(start);
  if (st != ECMC_OK) return st;
  // two rounds over the six axes: a later axis can change the best choice
  // on an earlier one (a round that changes nothing ends the search)
  for (int round = 0; round < 2; ++round) {
    const TunePoint before = cur;
    for (int axis = 0; axis < 6; ++axis) {
      const TunePoint base = cur;
      const int cnt = axis == 0 ? 4 : axis == 1 ? 7 : axis == 2 ? 2 : axis == 3 ? 4 : 3;
      for (int i = 0; i < cnt; ++i) {
        TunePoint pt = base;
        if (axis == 0) pt.lanes = lanes_c[i];
        if (axis == 1) pt.tile_side = tile_c[i];
        if (axis == 2) pt.cell_side = cell_c[i];
        if (axis == 3) pt.ecs = ecs_c[i];
        if (axis == 4) pt.warps = warps_c[i];
        if (axis == 5) pt.tight = tight_c[i];
        st = consider(pt);
        if (st != ECMC_OK) return st;
      }
    }
    if (round == 0 && before.lanes == cur.lanes && before.tile_side == cur.tile_side &&
        before.cell_side == cur.cell_side && before.ecs == cur.ecs && before.warps == cur.warps &&
        before.tight == cur.tight)
      break;
  }
  if (!have) return ECMC_EINVAL;
  *best = cur;
  *best_score = cur_s;
  *n_trials = n;
  return ECMC_OK;
}

}  // namespace ecmc
