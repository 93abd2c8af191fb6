/*
 * ecmc.h — C ABI of the GB300 event-chain Monte Carlo library for melts of
 * tethered hard-sphere bead chains.
 *
 * Method: Kampmann, Boltz, Kierfeld, "Monte Carlo Simulation of Dense Polymer
 * Melts Using Event Chain Algorithms" (arXiv:1502.06447).
 *   - EC move: Sec. II, the four-step rule (pick pivot and direction v; move
 *     the pivot by the largest admissible x <= x_max; hand the move to the
 *     limiting bead; repeat until x_max = 0), with the min-over-partners rule
 *     for several interaction partners (Sec. II).
 *   - Model: hard spheres of diameter sigma (Eq. 1) bonded into chains by
 *     tethers of maximal length b_max (Sec. II, model paragraph).
 *   - Parallel form: Sec. II.A — spatial tile-joint decomposition re-drawn
 *     every sweep, reflection of the EC at tile walls, and reflection of v at
 *     the plane normal to the bond when the bonded partner cannot move
 *     (Fig. 2c); the same reflection at a hard-sphere contact with a bead that
 *     cannot move.
 *   - Swap move: Sec. II.C (Fig. 4).
 *
 * Conventions (every entry point):
 *   - Returns an ecmc_status; never aborts.  ecmc_last_error() gives a
 *     one-line message for the calling thread's last failure.
 *   - Host buffers belong to the caller and are only read/written during the
 *     call.  Device memory belongs to the library (allocated in
 *     ecmc_create*, freed in ecmc_destroy).
 *   - Positions are interleaved xyz doubles, bead b at [3b, 3b+3), wrapped
 *     into [0, L).  Image counters are interleaved xyz int32; the unwrapped
 *     position is r + img * L.  Bead b belongs to chain b / N and is bonded to
 *     b-1 and b+1 of the same chain.
 *   - Work is issued on the context's stream (default: a stream the library
 *     creates; see ecmc_set_stream).  Calls that return host data
 *     synchronise that stream.
 *   - Device-side failures (event cap exceeded, a staging capacity exceeded)
 *     are recorded in a status word on the device and returned by the next
 *     call that synchronises.
 */
#ifndef ECMC_H
#define ECMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecmc_ctx ecmc_ctx;

typedef enum {
  ECMC_OK = 0,
  ECMC_EINVAL = -1,    /* bad argument */
  ECMC_ENOMEM = -2,    /* device allocation failed */
  ECMC_ECUDA = -3,     /* CUDA runtime error */
  ECMC_EOVERLAP = -4,  /* positions overlap (|r_ij| < sigma) */
  ECMC_ETETHER = -5,   /* a bond longer than b_max */
  ECMC_ESTUCK = -6,    /* an EC exceeded the event cap */
  ECMC_ECKPT = -7,     /* checkpoint file unreadable or inconsistent */
  ECMC_ECAPACITY = -8, /* a tile holds more beads than the staging buffer */
  ECMC_EBOUNDS = -9    /* bounds-checked build (-DECMC_CHECKED) only: a kernel
                          caught an index out of range, recorded the site and
                          skipped the access; results of that run are void */
} ecmc_status;

enum { ECMC_MODE_SERIAL = 0, ECMC_MODE_DOMAIN = 1 };
enum { ECMC_DIR_CART3 = 0, ECMC_DIR_ISO = 1 };
enum { ECMC_PREC_FP64 = 0, ECMC_PREC_FP32F = 1 };

/* event outcomes, also the order of ecmc_obs.events[] */
enum {
  ECMC_EV_END = 0,        /* x_max used up */
  ECMC_EV_PASS = 1,       /* free flight capped at s_cap; same pivot continues */
  ECMC_EV_WALL = 2,       /* tile wall: v's normal component flipped */
  ECMC_EV_HS_LIFT = 3,    /* hard-sphere contact, EC handed to the hit bead */
  ECMC_EV_HS_REFLECT = 4, /* contact with an immotile bead: v reflected */
  ECMC_EV_TE_LIFT = 5,    /* tether taut, EC handed to the bonded bead */
  ECMC_EV_TE_REFLECT = 6, /* tether taut, partner immotile: v reflected */
  ECMC_EV_SWAP = 7,       /* contact, swap accepted: same pivot continues */
  ECMC_NEV = 8
};

/* Run options.  Zero-initialise and set what you need; zero fields take
 * the defaults given. */
typedef struct ecmc_opts {
  int32_t mode;          /* ECMC_MODE_SERIAL (undecomposed) or _DOMAIN */
  int32_t dir_mode;      /* ECMC_DIR_CART3: v in {+x,+y,+z}; _ISO: uniform on S^2 */
  int32_t precision;     /* ECMC_PREC_FP64: every candidate in FP64;
                            _FP32F: FP32 screen + FP64 confirm (same events) */
  int32_t tiles[3];      /* tiles per axis D (domain mode); >= 3 */
  double joint;          /* joint width w (domain mode); 0 -> b_max; must be >= b_max */
  double s_cap;          /* longest single free flight; 0 -> 0.25 sigma */
  int64_t event_cap;     /* events per EC before ECMC_ESTUCK; 0 -> 10^7 */
  double p_swap;         /* swap proposal probability at a motile contact */
  int32_t ecs_per_tile;  /* ECs per tile per sweep (domain); 0 -> 1 */
  int32_t lanes;         /* lanes per EC: 32, 16, 8 or 4; 0 -> 32 */
  int32_t record;        /* 1: keep per-EC digests / lift sums of the last run */
  int32_t stage_cap;     /* staged beads per tile; 0 -> derived from the tile size */
  double cell_side;      /* side of the global cell grid (domain); 0 -> 1.05 sigma */
  double tile_side;      /* batch: target tile side when tiles[0] <= 0 (per replica
                            D = floor(L / tile_side), at least 3); 0 -> 4.2 sigma */
  int32_t schedule;      /* screened domain form with lanes 4, 8 or 16:
                            0 -> block lockstep: the tiles of a block advance one
                            event per step together and their FP64 work (candidate
                            evaluation, move) is packed one tile per thread;
                            1 -> warp lockstep: each group of `lanes` lanes does
                            its own tile's FP64 work.  Same events either way. */
  int32_t block_tiles;   /* block lockstep: tiles per block (a multiple of
                            32 / lanes, at most 32); 0 -> most tiles per SM */
  int32_t request_cap;   /* block lockstep: FP64 requests per tile and step in
                            the block's request list, 1..6; 0 -> 6.  A tile
                            whose FP32 survivors (or whose list of 24 x cap
                            screened slots) do not fit is evaluated
                            exhaustively in FP64 by its own lanes: same
                            events, slower; small caps exist to exercise that
                            path (ecmc_obs.exhaustive counts it). */
  double k_spring;       /* > 0: bead-spring chains (Sec. II): every bond is a
                            harmonic spring (k/2)(b - sigma)^2 with k =
                            k_spring in kT/sigma^2 (the paper's melts: 30)
                            instead of a tether; 0 -> tethers of b_max.  With
                            springs each bond of the pivot draws a Boltzmann
                            energy dE = -log(u) at every event (Philox tag 6,
                            counter (6 | ec << 8, sweep, unit, event), words 0
                            and 1 for the bonds to b - 1 and b + 1; serial
                            mode: ec = 0, sweep = 0, unit = the EC ordinal) and
                            its event is where the energy the move adds after
                            the closest approach reaches dE; a spring event
                            with a motile partner lifts, with an immotile one
                            reflects v at the plane normal to the bond
                            (Sec. II.A, Fig. 2c).  In the domain mode a bead
                            whose bonded bead is motile in another tile is
                            immotile for the sweep (springs have no longest
                            bond, so no joint could keep such tiles apart);
                            tether checks are off; swaps (p_swap > 0) and the
                            batch are refused. */
  double tight_factor;   /* block lockstep: the first launch of a sweep stages
                            tiles with capacities of tight_factor times a
                            melted tile's mean content (more tiles fit per SM);
                            tiles that do not fit run in a second launch with
                            the full capacities (same events); 0 -> 1.08 */
} ecmc_opts;

/* Observables and counters (Sec. IV observables; see ecmc_observables). */
typedef struct ecmc_obs {
  int64_t n_beads, n_chains, N;
  int64_t sweeps;              /* domain sweeps run so far */
  int64_t ecs;                 /* ECs run so far */
  int64_t events[ECMC_NEV];    /* event outcomes so far */
  int64_t events_total;
  int64_t swap_tried;
  double lift_sum;             /* sum over lifts of (r_target - r_pivot).v */
  double refl_sum;             /* same projection at immotile contacts */
  double disp_sum;             /* sum of all free flights (= ecs * ell) */
  double ell_sum;              /* sum of ell over ECs */
  double pressure;             /* betaP/rho = 1 + lift_sum / ell_sum: the
                                  lift-distance estimator; unbiased for
                                  serial runs, biased low in the domain mode
                                  (reflections and walls are not lifts) */
  double re2_mean;             /* <R_e^2> over chains (minimum-image bonds) */
  double bond_max, bond_min;   /* longest / shortest bond */
  int64_t overlaps;            /* pairs with |r_ij|^2 < sigma^2 (1 - 1e-10) */
  int64_t tether_violations;   /* bonds with b^2 > b_max^2 (1 + 1e-10) */
  double g1;                   /* middle-bead MSD vs the reference snapshot */
  double device_seconds;       /* device time of all ecmc_run calls */
  double ec_kernel_seconds;    /* device time of the EC kernel launches alone */
  int64_t confirmed;           /* FP64 confirmations of the FP32 screen */
  /* contact values of the current state (virial theorem for hard
   * constraints, valid whatever moves produced the state), shell width
   * d = contact_delta: */
  int64_t contact_pairs[2];    /* pairs with |r_ij| in [sigma, sigma + d), [sigma + d, sigma + 2d) */
  int64_t taut_bonds[2];       /* bonds in (b_max - d, b_max], (b_max - 2d, b_max - d] */
  double contact_delta;        /* d = 0.02 sigma */
  double pressure_contact;     /* betaP/rho = 1 + [sigma f(sigma+) - b_max f_b(b_max-)] / (3 n),
                                  f, f_b pairs / bonds per unit distance at
                                  contact, each extrapolated linearly from its
                                  two shells */
  int64_t exhaustive;          /* tile steps of the block-lockstep kernel
                                  evaluated exhaustively in FP64 */
  double bond_mean;            /* <b> over all bonds of the current state */
} ecmc_obs;

/* One EC event of the parity log (ecmc_event_log). */
typedef struct ecmc_event {
  int64_t unit;      /* EC ordinal within the last run */
  int32_t seq;       /* event index within the EC */
  int32_t pivot;     /* pivot bead id before the event */
  int32_t kind;      /* ECMC_EV_* */
  int32_t pad;
  int64_t partner;   /* bead id, wall axis, or -1 */
  double x;          /* free flight of the pivot */
} ecmc_event;

/* Phantom chains (Sec. II.B, the first stage of the paper's initial
 * configurations: chains without excluded volume, to be pushed apart
 * afterwards).  n_chains non-reversal random walks of N beads with bond
 * length `bond` in the periodic box L: the first bead uniform in the box,
 * the first bond uniform on the sphere, every next bond uniform on the cap
 * t_j . t_{j+1} >= cos(theta_max) = (c - 3)/(c + 1) around the one before,
 * so that <cos theta> = (c - 1)/(c + 1) and <R^2> -> c (N - 1) bond^2 for
 * long chains (c = 1: free random walk; the paper's melts have c = 1.9).
 * Philox4x64-10 with key (seed, 0), counter (5, chain, bead, attempt); the
 * azimuth comes from the first point of the unit disc among uniform points
 * of the square (at most 256 attempts, else ECMC_EINVAL).  xyz_out (host,
 * 3 n_chains N doubles) receives positions wrapped into [0, L), img_out
 * (host, 3 n_chains N int32, or NULL) the image counters.  Needs c >= 1,
 * bond > 0.  Allocates and frees device memory; synchronises. */
ecmc_status ecmc_phantom_chains(const double L[3], int64_t n_chains, int32_t N, double bond,
                                double c, uint64_t seed, double *xyz_out, int32_t *img_out);

/* Slow push-off (Sec. II.B).  ecmc_create_phantom makes a context whose
 * beads are phantom chains (as ecmc_phantom_chains: n_chains x N beads,
 * bond length `bond` <= b_max, stiffness c, key (seed, 0)) in the periodic
 * box; they may overlap, so ecmc_run refuses it (ECMC_EOVERLAP) until
 * ecmc_pushoff (or a valid ecmc_set_positions) has resolved it.
 * ecmc_pushoff grows the hard-sphere diameter from f0 sigma to sigma in
 * `stages` equal steps, d_k = sigma (f0 + (1 - f0) k / stages), d_stages =
 * sigma; at every diameter it repeats domain sweeps (the configured tiles;
 * needs the domain mode, ECMC_PREC_FP64 and 4-32 lanes) in which every tile
 * runs one EC of length ell from each of its motile beads that overlaps
 * another bead (|r_ij|^2 < d^2 (1 - 1e-10)), in bead id order, with the
 * direction draw of EC e as in ecmc_run and the pivot ignoring the beads it
 * overlaps, until no overlap is left.  With bead springs configured
 * (k_spring > 0) the springs act during the push-off with rest length d, the
 * current diameter (every length of the model grows together).  Sweeps
 * continue the context's sweep count (Philox counters as in ecmc_run with
 * `seed`); swaps are off.
 * *sweeps_out (may be NULL) receives the sweeps run.  ECMC_ESTUCK if a
 * diameter is not resolved within max_sweeps sweeps; the final state is
 * checked as ecmc_set_positions checks it. */
ecmc_status ecmc_create_phantom(const double box[3], int64_t n_chains, int32_t N, double bond,
                                double stiffness, uint64_t seed, double sigma, double b_max,
                                ecmc_ctx **out);
ecmc_status ecmc_pushoff(ecmc_ctx *ctx, double f0, int32_t stages, double ell, uint64_t seed,
                         int64_t max_sweeps, int64_t *sweeps_out);

/* ---- creation ----------------------------------------------------------
 * ecmc_create_lattice: melt on an n0 x n1 x n2 simple-cubic lattice with
 * spacing a in a periodic box L = dims * a.  Sites are visited in a 3-D
 * snake (x fastest, reversing every row; y reversing every plane) and cut
 * into consecutive runs of N beads = chains, so every bond is one lattice
 * step (requires sigma <= a <= b_max and N | n0 n1 n2).  Each coordinate is
 * moved by jitter*(2u-1), u from Philox4x64-10 with key (seed, 0) and counter
 * (4, 0, bead, 0), words 0..2 for x..z; jitter 0 keeps the exact lattice.
 * (The paper builds melts by random-walk growth and push-off, Sec. II.B; the
 * lattice start is a synthetic stand-in.)  Checks the start for overlaps
 * and tether violations (ECMC_EOVERLAP / ECMC_ETETHER).  *out receives the
 * context. */
ecmc_status ecmc_create_lattice(const int32_t dims[3], double spacing,
                                double jitter, uint64_t seed, int32_t N,
                                double sigma, double b_max, ecmc_ctx **out);

/* ecmc_create: melt of n_chains chains of N beads at volume fraction phi.
 * box: NULL or {0,0,0} -> a cube with phi = n pi sigma^3 / (6 V); otherwise
 * the box must agree with phi within 1e-3 relative.  The beads are placed
 * on the lattice of ecmc_create_lattice whose dims are the factorisation of
 * n_chains*N closest to the box shape (jitter 0.01 sigma, seed 0). */
ecmc_status ecmc_create(const double box[3], double phi, int32_t n_chains,
                        int32_t N, double sigma, double b_max, ecmc_ctx **out);

void ecmc_destroy(ecmc_ctx *ctx);
const char *ecmc_last_error(void);

/* Use this CUDA stream (a cudaStream_t passed as void*) for all work of the
 * context; NULL restores the library's own stream. */
ecmc_status ecmc_set_stream(ecmc_ctx *ctx, void *stream);

/* ---- state --------------------------------------------------------------
 * xyz: host, 3n doubles (caller-owned; pinned memory is copied fastest).
 * set: wraps into [0,L) on the device, adding whole boxes to the image
 * counters (which start from img, 3n int32, or 0 when img is NULL), then
 * checks non-finite coordinates (ECMC_EINVAL), overlaps and tethers; after
 * a failed set the context's state is undefined until a successful one. */
ecmc_status ecmc_set_positions(ecmc_ctx *ctx, const double *xyz,
                               const int32_t *img);
ecmc_status ecmc_get_positions(ecmc_ctx *ctx, double *xyz_out,
                               int32_t *img_out /* may be NULL */);
/* box, bead count, chain length */
ecmc_status ecmc_get_info(ecmc_ctx *ctx, double box[3], int64_t *n_beads,
                          int32_t *N);

/* ---- running ------------------------------------------------------------ */
ecmc_status ecmc_configure(ecmc_ctx *ctx, const ecmc_opts *opts);

/* ecmc_run: serial mode: chains_per_sweep ECs (all of them, n_sweeps is
 * ignored), EC j of the context's lifetime starting at a uniform bead with
 * Philox counter (1, 0, j, attempt).  Domain mode: n_sweeps sweeps; in
 * sweep s the tile shift comes from Philox counter (2, s, 0, 0) and every
 * tile holding motile beads runs ecs_per_tile ECs (chains_per_sweep <= 0
 * keeps opts.ecs_per_tile, > 0 overrides it).  Each EC has total displacement
 * ell.  Sweeps and ECs continue the context's counters, so a run split in
 * two calls equals one call. */
ecmc_status ecmc_run(ecmc_ctx *ctx, double ell, int64_t chains_per_sweep,
                     uint64_t seed, int64_t n_sweeps);

/* Swap moves (Sec. II.C).  Sets p_swap so that the swap attempts per bead
 * per sweep match the target, from the motile hard-sphere contacts counted
 * during the last ecmc_run call (contacts are counted with or without
 * swaps: each one lifts or swaps; run on the state and launch setting to be
 * calibrated; push-off, autotuning and restore start no such run):
 * p_swap = min(1, target * n_beads * sweeps / contacts), with sweeps and
 * contacts of that run.  target 0 disables swaps.  ECMC_EINVAL
 * when no run with contacts came before. */
ecmc_status ecmc_swap(ecmc_ctx *ctx, double attempts_per_bead_per_sweep);

/* Fused observables over the current state (R_e^2, bonds, overlaps, g1)
 * together with the counters of all runs so far.  Synchronises. */
ecmc_status ecmc_observables(ecmc_ctx *ctx, ecmc_obs *out);
/* take the g1 reference snapshot (unwrapped middle beads) now; also the
 * g2 reference of ecmc_structure (middle beads relative to their chain's
 * centre of mass) */
ecmc_status ecmc_g1_reset(ecmc_ctx *ctx);

/* g1 table (Sec. IV, Eq. 3: g1(dt) = <[r_{N/2}(t + dt) - r_{N/2}(t)]^2>_t,
 * averaged over the chains and over time origins t), accumulated on the
 * device after every domain sweep of ecmc_run from this call on.  Lags are
 * log-spaced, dt = j P^k sweeps for k = 0 .. K-1 and j = 1 .. P-1 (so lags
 * up to (P - 1) P^(K-1)); the origins of lag j P^k are the sweeps that are
 * multiples of P^k (counted from this call, whose state is sweep 0) with
 * t + dt within the run.  Positions are the unwrapped middle beads
 * (bead N/2 of each chain, r + img L).  The device keeps K rings of P
 * snapshots (K P 24 B per chain) and one sum and count per lag; the sum
 * for a lag adds, sweep by sweep, the chains' (dx^2 + dy^2) + dz^2 in chain
 * order, so it is reproducible bit for bit.  ecmc_g1_track(ctx, P, K)
 * (2 <= P <= 64, 1 <= K <= 16) starts a new table; P = 0 stops tracking
 * (the table is kept).  Serial runs leave the table unchanged. */
ecmc_status ecmc_g1_track(ecmc_ctx *ctx, int32_t P, int32_t K);
/* lag (sweeps), g1 (sigma^2; 0 where a lag has no origin yet) and the
 * number of origins per lag, K (P - 1) entries in order k = 0.. , j = 1..
 * (host buffers of at least cap entries, any may be NULL); *n receives the
 * entries written.  Synchronises. */
ecmc_status ecmc_g1_table(ecmc_ctx *ctx, int64_t *lag, double *g1, int64_t *count, int32_t cap,
                          int32_t *n);

/* Chain structure of the current state (one fused pass, Sec. IV: radius of
 * gyration and g2; Appendix A: moment of inertia tensor and shape
 * descriptors, end-to-end distance distribution W(R); Sec. II.B: internal
 * distances R^2(n)).  Positions along a chain come from minimum-image bonds
 * (u_0 = 0, u_{j+1} = u_j + minimg(r_{j+1} - r_j)); the gyration tensor is
 * S = (1/N) sum_j (u_j - U)(u_j - U)^T with U = (1/N) sum_j u_j, and the
 * moment of inertia tensor N (Tr S 1 - S): taken in descending order its
 * eigenvalues give <I1 + I2 - I3> / <Tr I> = lam_sum[2] / rg2_sum,
 * <I1 - I2 + I3> / <Tr I> = lam_sum[1] / rg2_sum,
 * <-I1 + I2 + I3> / <Tr I> = lam_sum[0] / rg2_sum and
 * <4 b_I^2 + 3 c_I^2> / <Tr I>^2 = n_chains bc_sum / (4 rg2_sum^2).  Sums
 * run over chains in chain order and are reproducible bit for bit; the
 * eigenvalues come from a Jacobi iteration (within 1e-14 Tr S of exact). */
typedef struct ecmc_struct {
  int64_t n_chains, N;
  double rg2_sum;     /* sum over chains of R_g^2 = Tr S */
  double lam_sum[3];  /* sums of the eigenvalues of S, lam1 <= lam2 <= lam3 per chain */
  double b_sum;       /* asphericity lam3 - (lam1 + lam2) / 2 */
  double c_sum;       /* acylindricity lam2 - lam1 */
  double kappa2_sum;  /* shape anisotropy 1 - 3 P / (Tr S)^2, P = lam1 lam2 + lam2 lam3 + lam3 lam1 */
  double bc_sum;      /* 4 b^2 + 3 c^2 = 4 ((Tr S)^2 - 3 P) */
  double g2_sum;      /* |m - m_ref|^2, m = u_{N/2} - U, m_ref from the last
                         ecmc_g1_reset (0 without one) */
  double re2_sum;     /* |u_{N-1}|^2 */
} ecmc_struct;
/* r2n: NULL or N doubles (host), receives R^2(n) = mean over chains and j of
 * |u_{j+n} - u_j|^2 for n < N (r2n[0] = 0); hist: NULL or nbins int64
 * (host), receives the chains with floor(|u_{N-1}| / dR) = b (the last bin
 * takes the rest; dR > 0).  Needs chains of at least 2 beads.  Device
 * scratch (about 24 B per bead, plus 8 B per bead for R^2(n)) is allocated
 * on first use.  Synchronises. */
ecmc_status ecmc_structure(ecmc_ctx *ctx, ecmc_struct *out, double *r2n, double dR,
                           int64_t nbins, int64_t *hist);

/* Per-EC records of the last ecmc_run (opts.record = 1): digest (64-bit
 * FNV-1a over (pivot, kind<<32|partner, bits of x) of every event), lift sum
 * and event count, in EC ordinal order: serial -> EC order; domain ->
 * ((sweep * n_tiles) + tile) * ecs_per_tile + ec, tiles without motile
 * beads left at digest 0.  Buffers hold at least *n entries on input
 * (caller-owned host memory); *n receives the count. */
ecmc_status ecmc_records(ecmc_ctx *ctx, uint64_t *digest, double *lift,
                         int64_t *events, int64_t *n);
/* Event log of the last run (opts.record = 1, capacity from ecmc_log_reserve),
 * unordered across ECs; sort by (unit, seq). */
ecmc_status ecmc_log_reserve(ecmc_ctx *ctx, int64_t cap);
ecmc_status ecmc_event_log(ecmc_ctx *ctx, ecmc_event *buf, int64_t cap,
                           int64_t *n);

/* Domain assignment of sweep `sweep` for the current positions: tile of
 * each bead (-1 = joint) and the shift.  tags: n int32, shift: 3 doubles. */
ecmc_status ecmc_domain_tags(ecmc_ctx *ctx, uint64_t seed, int64_t sweep,
                             int32_t *tags, double shift[3]);

/* ---- checkpoint ---------------------------------------------------------
 * Binary file: header (magic, version, sizes), positions, images, counters,
 * opts, and a checksum.  Because every random number is a function of
 * (seed, sweep/EC counter), restore + run equals an uninterrupted run. */
ecmc_status ecmc_checkpoint(ecmc_ctx *ctx, const char *path);
ecmc_status ecmc_restore(ecmc_ctx *ctx, const char *path);

/* ---- batched replicas ------------------------------------------------------
 * Many independent melts advanced together: per sweep one domain assignment +
 * cell list pass over all replicas' beads and one EC launch over all
 * replicas' tiles (the Sec. II.A sweep of each replica), optionally captured
 * once in a CUDA graph and replayed (the sweep counter lives on the device).
 * Replica r is the lattice melt of ecmc_create_lattice with dims, spacing, N
 * of specs[r] and jitter, and draws every random number with the Philox key
 * (seed, r): it evolves exactly as a single melt with that key would.  All
 * replicas share sigma and b_max.  Positions are concatenated in replica
 * order. */
typedef struct ecmc_replica_spec {
  int32_t dims[3];
  double spacing;
  int32_t N;
  double sigma, b_max;
} ecmc_replica_spec;
typedef struct ecmc_batch ecmc_batch;
ecmc_status ecmc_batch_create(const ecmc_replica_spec *specs, int32_t n,
                              double jitter, uint64_t seed, ecmc_batch **out);
void ecmc_batch_destroy(ecmc_batch *b);
/* opts as for ecmc_configure, domain mode only; tiles[0] <= 0 -> per
 * replica tiles from opts.tile_side; lanes 4, 8, 16 or 32 (0 -> 8). */
ecmc_status ecmc_batch_configure(ecmc_batch *b, const ecmc_opts *opts);
/* n_sweeps sweeps of every replica; use_graph = 1 captures one sweep in a
 * CUDA graph (after one uncaptured sweep) and replays it. */
ecmc_status ecmc_batch_run(ecmc_batch *b, double ell, uint64_t seed,
                           int64_t n_sweeps, int32_t use_graph);
/* replica r's positions / images (host buffers of 3 n_r entries) */
ecmc_status ecmc_batch_get_positions(ecmc_batch *b, int32_t replica,
                                     double *xyz_out, int32_t *img_out);
/* replica r's tiles per axis, first unit in the concatenated tile
 * numbering, bead count (any output may be NULL) */
ecmc_status ecmc_batch_info(ecmc_batch *b, int32_t replica, int32_t tiles[3],
                            int64_t *unit_off, int64_t *n_beads);
ecmc_status ecmc_batch_stats(ecmc_batch *b, int64_t *events_total,
                             int64_t *ecs, double *device_seconds);
/* per-EC records of the last run (opts.record = 1), ordered as
 * ((sweep * units) + unit) * ecs_per_tile + ec over the concatenated units */
ecmc_status ecmc_batch_records(ecmc_batch *b, uint64_t *digest, double *lift,
                               int64_t *events, int64_t *n);

/* ---- autotuner -------------------------------------------------------------
 * Picks the launch setting of the domain sweep for this machine and system
 * (the paper fixes none: Sec. II.A leaves the tile size open): lanes per EC
 * (4, 8, 16, 32), tile side (3.4, 3.8, 4.2, 4.6, 5, 6, 7 sigma), global cell side (1.05 or 1.4
 * sigma), ECs per tile (1, 2, 4 or 8) and the block-lockstep kernel's staging
 * (1, 2 or 4 warps per block; first-pass capacity factor 1.0, 1.08 or 1.16;
 * other kernels take only the defaults), by a coordinate descent (up to two
 * rounds) over short timed trials.  Each trial restores the state saved on entry, runs one untimed
 * sweep and `trial_sweeps` timed ones; the score is ECs per device-second.
 * On return the context (batch) is configured with the winner and its
 * positions, images, counters, sums and sweep index are those on entry, so a
 * run after tuning is the run that would have followed without it (with the
 * winner's tiles).  Needs a configured domain-mode context; keeps its mode,
 * direction rule, precision, p_swap, joint, s_cap and record setting. */
typedef struct ecmc_tuning {
  int32_t lanes;          /* lanes per EC */
  double tile_side;       /* target tile side (sigma) */
  double cell_side;       /* global cell side (sigma) */
  int32_t ecs_per_tile;
  int32_t tiles[3];       /* single context: tiles per axis; batch: 0 */
  double ecs_per_s;       /* score of the winner */
  double events_per_s;
  int32_t n_trials;       /* admissible points timed */
  int32_t block_tiles;    /* block lockstep: tiles per block (0: not that kernel) */
  double tight_factor;    /* block lockstep: first-pass capacity factor */
} ecmc_tuning;
ecmc_status ecmc_autotune(ecmc_ctx *ctx, double ell, uint64_t seed,
                          int32_t trial_sweeps, ecmc_tuning *out);
ecmc_status ecmc_batch_autotune(ecmc_batch *b, double ell, uint64_t seed,
                                int32_t trial_sweeps, ecmc_tuning *out);

/* ---- domain assignment and cell list without allocation ------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory (a host callback, a framework that owns every
 * device allocation, a real-time loop that must stay off the driver's
 * allocator).  It computes what a sweep's first step computes — the tile of
 * every bead for sweep `sweep` (-1 = joint; shift from Philox counter
 * (2, sweep, 0, 0), key (seed, 0); tiles[a] tiles of width box[a]/tiles[a]
 * along axis a, the last `joint` of each being joint) and the beads binned
 * into the cell grid nc_a = floor(box[a] / cell_side) — into buffers the
 * caller owns, and calls no cudaMalloc, cudaFree or allocating routine.
 *   d_r          device, 3n doubles, positions wrapped into [0, box)
 *   d_tags       device, n int32 (out)
 *   d_cell_start device, ncell + 1 int32 (out), ncell = nc_0 nc_1 nc_2;
 *                cell c = (z nc_1 + y) nc_0 + x holds d_cell_ids[start[c],
 *                start[c+1]) (order inside a cell not fixed)
 *   d_cell_ids   device, n int32 (out)
 *   shift_out    host, 3 doubles (out) or NULL
 *   stream       cudaStream_t as void*, NULL for the default stream
 * Limits: n <= 1,048,576 beads and ncell <= 1,048,576 cells; larger inputs
 * return ECMC_EINVAL.  Scratch: an 8 MiB file-scope __device__ array that
 * every GPU that loads the library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * with the device current; make that first call before any stream capture.
 * The address is kept for the life of the process: after a cudaDeviceReset
 * of that device it is stale, and this entry point must not be called again
 * in that process.  Arguments are checked before any launch: box and cell
 * side must give at most 1,048,576 cells per axis and in total, and the
 * tiles at most 2^31 - 1 in total (ECMC_EINVAL otherwise).  A CUDA failure
 * returns ECMC_ECUDA with the CUDA error in ecmc_last_error().
 * All calls share the array and it keeps the last call's contents (the
 * counts are cleared by each call); calls whose work overlaps on the GPU
 * race and must be serialised by the caller.  Asynchronous on `stream`. */
ecmc_status ecmc_cells_static(const double *d_r, int64_t n, const double box[3],
                              const int32_t tiles[3], double joint,
                              double cell_side, uint64_t seed, int64_t sweep,
                              int32_t *d_tags, int32_t *d_cell_start,
                              int32_t *d_cell_ids, double shift_out[3],
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif
