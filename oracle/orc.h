/*
 * Oracle for the event-chain (EC) Monte Carlo move of tethered hard-sphere
 * bead chains (Kampmann, Boltz, Kierfeld, "Monte Carlo Simulation of Dense
 * Polymer Melts Using Event Chain Algorithms", arXiv:1502.06447).
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, serial, FP64 C code is the checker
 * of the CUDA path.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no code with the CUDA
 * library: its own Philox, its own geometry, its own cell list.
 *
 * Layout: positions are interleaved xyz doubles, wrapped into [0,L); image
 * counters are interleaved xyz int32 (unwrapped = r + img*L).  Bead b of a
 * system with chains of N beads belongs to chain b/N and is bonded to b-1 and
 * b+1 inside that chain (chains are consecutive id runs).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

enum { ORC_SERIAL = 0, ORC_DOMAIN = 1 };
enum { ORC_DIR_CART3 = 0, ORC_DIR_ISO = 1, ORC_DIR_PLUSX = 2 };

/* candidate kinds, in tie-break order (smaller wins an exact tie) */
enum { K_END = 0, K_PASS = 1, K_WALL = 2, K_HS = 3, K_TETHER = 4 };

/* outcome counters */
enum {
  O_END = 0, O_PASS, O_WALL, O_HS_LIFT, O_HS_REFLECT,
  O_TE_LIFT, O_TE_REFLECT, O_SWAP, O_NOUT
};

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ESTUCK = -6, ORC_ETILE = -8 };

typedef struct {
  int64_t n;          /* number of beads */
  int32_t N;          /* beads per chain (1 = unbonded spheres) */
  int32_t mode;       /* ORC_SERIAL or ORC_DOMAIN */
  double L[3];        /* periodic box */
  double sigma;       /* hard-sphere diameter */
  double b_max;       /* tether length */
  double s_cap;       /* longest single free flight (pass event beyond) */
  int32_t dir_mode;   /* ORC_DIR_* */
  int32_t D[3];       /* tiles per axis (domain mode) */
  double w;           /* joint width (domain mode) */
  double p_swap;      /* swap proposal probability at a motile contact */
  int64_t event_cap;  /* events per EC before ORC_ESTUCK */
  int32_t use_cells;  /* 1: own cell list, 0: all-pairs search */
  int32_t ecs_per_tile;
  uint64_t seed;
  uint64_t replica;
  /* slow push-off (Sec. II.B): ECs start at the flagged motile beads of a
   * tile (one each, in bead id order) and a pivot ignores the beads it
   * overlaps */
  int32_t pushoff;
  int32_t pad_po;
  const uint8_t *po_flag;
  /* k > 0: bonds are harmonic springs (k/2)(b - sigma)^2 (Sec. II, bead-
   * spring chains, k in units of kT/sigma^2) instead of tethers; b_max is
   * then unused and swaps are off */
  double k_spring;
  /* domain mode, work split for timing on several host cores: only tiles
   * t with t % tile_mod == tile_rem run (tile_mod <= 1: all tiles); tiles
   * are independent within a sweep, so each part is exactly the serial
   * oracle's work on those tiles */
  int32_t tile_mod, tile_rem;
} orc_params;

typedef struct {
  int64_t ecs;
  int64_t events;
  int64_t out[O_NOUT];
  int64_t swap_tried;
  double lift_sum;    /* sum over lifts of (r_target - r_pivot).v */
  double refl_sum;    /* same projection, immotile contacts (reported apart) */
  double disp_sum;    /* sum of all free flights */
  int64_t status;
} orc_stats;

typedef struct {
  int64_t unit;       /* EC ordinal within the call */
  int32_t pivot;
  int32_t kind;       /* outcome O_* */
  int64_t partner;
  double x;
} orc_event;

#endif
