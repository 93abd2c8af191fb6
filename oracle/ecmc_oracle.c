/*
 * Oracle for the event-chain Monte Carlo move of tethered hard-sphere chains
 * (arXiv:1502.06447).  TEST INFRASTRUCTURE ONLY: see orc.h.
 *
 * What it follows:
 *   - EC move, Sec. II (the four-step rule): pick pivot and direction v, move
 *     the pivot by the largest admissible x <= x_max, hand the move to the
 *     bead that limits it, repeat until x_max = 0.
 *   - Min-over-partners rule, Sec. II: with several interaction partners the
 *     admissible displacement is the minimum over partners and the chain is
 *     continued at the partner realising it.  For tethers of length b_max
 *     (Sec. II, model paragraph) the partner limit is where the bond becomes
 *     taut; hard spheres (Eq. 1) limit at contact.
 *   - Parallelisation, Sec. II.A: a spatial decomposition re-drawn every
 *     sweep, tile-joint partition, reflection of the EC at cell walls and, for
 *     a bond partner that cannot move, reflection of v at the plane normal to
 *     the bond (Fig. 2c); the same reflection at a hard-sphere contact with a
 *     bead that cannot move.
 *   - Swap move, Sec. II.C: at hard-sphere contact a swap of the two touching
 *     beads is proposed and accepted by Metropolis (infinite tether walls:
 *     accept iff every bond stays <= b_max); accepted -> beads exchanged and
 *     the same pivot continues; rejected -> ordinary transfer.
 *   - ECs with pair potentials, Sec. II (Fig. 2b): bead-spring chains, each
 *     bond drawing a Boltzmann energy per event that the pivot's move may
 *     spend where the bond energy rises.
 *   - Initial configurations, Sec. II.B: phantom chains grown as
 *     non-reversal random walks, then the slow push-off (ECs started at
 *     overlapping beads that ignore their pivot's overlaps, the diameter
 *     grown in stages).
 *   - Chain structure, Sec. IV and Appendix A: gyration tensor and centre
 *     of mass, internal distances R^2(n), end-to-end distance histogram.
 * Readings where the paper is silent (the tie order, the pass event, the
 * random-number layout, the joint width) are the same as the CUDA library's
 * and are written out at each place below.
 *
 * Compiled with -O2 -ffp-contract=off: every FP64 expression is evaluated
 * exactly as written, in IEEE round-to-nearest; multiply-adds are fused only
 * where written as fma() (C99, one rounding): the dot products and squared
 * lengths of the event geometry, the position update and the reflection.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "orc.h"

/* ---------------------------------------------------------------------
 * Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Round: two 64x64->128 products of the even
 * counter words with the round multipliers, the high halves xor-ed with the
 * odd words and the key, words permuted; the key is bumped by the Weyl
 * constants between rounds.
 * ------------------------------------------------------------------- */
#define PH_M0 0xD2E7470EE14C6C93ULL
#define PH_M1 0xCA5A826395121157ULL
#define PH_W0 0x9E3779B97F4A7C15ULL
#define PH_W1 0xBB67AE8584CAA73BULL

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                       uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    unsigned __int128 p0 = (unsigned __int128)PH_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PH_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += PH_W0;
    k1 += PH_W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* random-number layout (a reading; the paper fixes none):
 *   key  = (seed, replica)
 *   ctr  = (tag | ec<<8, sweep, unit, attempt)
 *   tag 1: start bead + direction; tag 2: domain shift; tag 3: swap draws */
enum { TAG_START = 1, TAG_SHIFT = 2, TAG_SWAP = 3, TAG_SPRING = 6 };

static void draw(const orc_params *P, uint64_t tag, uint64_t sweep,
                 uint64_t unit, uint64_t attempt, uint64_t out[4]) {
  uint64_t ctr[4] = {tag, sweep, unit, attempt};
  uint64_t key[2] = {P->seed, P->replica};
  orc_philox4x64_10(ctr, key, out);
}

/* uniform double in [0,1) from the top 53 bits */
static double u53(uint64_t w) { return (double)(w >> 11) * 0x1.0p-53; }

/* floor(w * m / 2^64): uniform integer in [0, m) */
static int64_t below(uint64_t w, int64_t m) {
  return (int64_t)(((unsigned __int128)w * (uint64_t)m) >> 64);
}

/* ---------------------------------------------------------------------
 * geometry
 * ------------------------------------------------------------------- */
static double minimg(double d, double L) {
  double h = 0.5 * L;
  if (d > h) d -= L;
  else if (d < -h) d += L;
  return d;
}

/* r += x v on one axis, then back into [0,L) with the image counter */
static void advance(double *r, int32_t *img, double x, double v, double L) {
  double y = fma(x, v, *r);
  if (y >= L) {
    y -= L;
    *img += 1;
  } else if (y < 0.0) {
    y += L;
    *img -= 1;
    if (y >= L) { /* -tiny + L rounded up to L */
      y = 0.0;
      *img += 1;
    }
  }
  *r = y;
}

/* ---------------------------------------------------------------------
 * state
 * ------------------------------------------------------------------- */
typedef struct {
  orc_params P;
  double *r;       /* 3n */
  int32_t *img;    /* 3n */
  /* own cell list (doubly linked, always current) */
  int nc[3];
  double cs[3];
  int32_t *head, *next, *prev, *cell;
  /* domain mode */
  int32_t *tag;    /* tile of each bead this sweep, -1 = joint */
  double shift[3], T[3], W[3];
  /* output */
  orc_stats *st;
  orc_event *log;
  int64_t log_cap, *log_n;
  uint64_t *digest;   /* per EC, or NULL */
  double *ec_lift;    /* per EC lift sum, or NULL */
  int64_t *ec_events; /* per EC event count, or NULL */
} ctx_t;

static int cell_of(const ctx_t *c, int64_t b) {
  int id[3];
  for (int a = 0; a < 3; ++a) {
    int k = (int)(c->r[3 * b + a] / c->cs[a]);
    if (k >= c->nc[a]) k = c->nc[a] - 1;
    if (k < 0) k = 0;
    id[a] = k;
  }
  return (id[2] * c->nc[1] + id[1]) * c->nc[0] + id[0];
}

static void cell_insert(ctx_t *c, int64_t b, int ci) {
  c->cell[b] = ci;
  c->prev[b] = -1;
  c->next[b] = c->head[ci];
  if (c->head[ci] >= 0) c->prev[c->head[ci]] = (int32_t)b;
  c->head[ci] = (int32_t)b;
}

static void cell_remove(ctx_t *c, int64_t b) {
  int ci = c->cell[b];
  if (c->prev[b] >= 0) c->next[c->prev[b]] = c->next[b];
  else c->head[ci] = c->next[b];
  if (c->next[b] >= 0) c->prev[c->next[b]] = c->prev[b];
}

static void cell_update(ctx_t *c, int64_t b) {
  if (!c->P.use_cells) return;
  int ci = cell_of(c, b);
  if (ci != c->cell[b]) {
    cell_remove(c, b);
    cell_insert(c, b, ci);
  }
}

static int ctx_init(ctx_t *c, const orc_params *P, double *r, int32_t *img) {
  memset(c, 0, sizeof(*c));
  c->P = *P;
  c->r = r;
  c->img = img;
  if (c->P.use_cells) {
    /* cell side >= (s_cap + sigma)(1 + 1e-9): every bead that can be hit
     * within one free flight sits in the 27 cells around the pivot */
    double reach = (P->s_cap + P->sigma) * (1.0 + 1e-9);
    int64_t ncell = 1;
    for (int a = 0; a < 3; ++a) {
      c->nc[a] = (int)floor(P->L[a] / reach);
      if (c->nc[a] < 3) {
        c->P.use_cells = 0;
        break;
      }
      c->cs[a] = P->L[a] / c->nc[a];
      ncell *= c->nc[a];
    }
    if (c->P.use_cells) {
      c->head = (int32_t *)malloc(sizeof(int32_t) * ncell);
      c->next = (int32_t *)malloc(sizeof(int32_t) * P->n);
      c->prev = (int32_t *)malloc(sizeof(int32_t) * P->n);
      c->cell = (int32_t *)malloc(sizeof(int32_t) * P->n);
      for (int64_t i = 0; i < ncell; ++i) c->head[i] = -1;
      for (int64_t b = P->n - 1; b >= 0; --b) cell_insert(c, b, cell_of(c, b));
    }
  }
  c->tag = (int32_t *)malloc(sizeof(int32_t) * (P->n > 0 ? P->n : 1));
  for (int64_t b = 0; b < P->n; ++b) c->tag[b] = 0;
  return ORC_OK;
}

static void ctx_free(ctx_t *c) {
  free(c->head);
  free(c->next);
  free(c->prev);
  free(c->cell);
  free(c->tag);
}

/* ---------------------------------------------------------------------
 * candidate search
 * ------------------------------------------------------------------- */
typedef struct {
  double x;
  int kind;
  int64_t partner;
  double dv; /* (r_pivot - r_partner).v before the flight (contact, tether) */
} cand_t;

static void consider(cand_t *best, double x, int kind, int64_t partner, double dv) {
  if (x < best->x ||
      (x == best->x &&
       (kind < best->kind || (kind == best->kind && partner < best->partner)))) {
    best->x = x;
    best->kind = kind;
    best->partner = partner;
    best->dv = dv;
  }
}

/* hard-sphere contact distance of pivot i moving along v towards bead k
 * (Eq. 1: contact at |r_i + x v - r_k| = sigma); returns -1 if none */
static double hs_dist(const ctx_t *c, int64_t i, int64_t k, const double v[3],
                      double *dv_out) {
  const double *L = c->P.L;
  double d0 = minimg(c->r[3 * i + 0] - c->r[3 * k + 0], L[0]);
  double d1 = minimg(c->r[3 * i + 1] - c->r[3 * k + 1], L[1]);
  double d2 = minimg(c->r[3 * i + 2] - c->r[3 * k + 2], L[2]);
  double dv = fma(d2, v[2], fma(d1, v[1], d0 * v[0]));
  *dv_out = dv;
  if (!(dv < 0.0)) return -1.0;
  double dd = fma(d2, d2, fma(d1, d1, d0 * d0));
  double sig2 = c->P.sigma * c->P.sigma;
  /* push-off: a bead the pivot overlaps is no obstacle (Sec. II.B) */
  if (c->P.pushoff && dd < sig2) return -1.0;
  double disc = sig2 - fma(-dv, dv, dd);
  if (!(disc > 0.0)) return -1.0;
  double x = -dv - sqrt(disc);
  if (x < 0.0) x = 0.0;
  return x;
}

/* tether limit of pivot i bonded to j: |r_i + x v - r_j| = b_max, the
 * positive root (the bond can always shorten first) */
static double te_dist(const ctx_t *c, int64_t i, int64_t j, const double v[3],
                      double *dv_out) {
  const double *L = c->P.L;
  double d0 = minimg(c->r[3 * i + 0] - c->r[3 * j + 0], L[0]);
  double d1 = minimg(c->r[3 * i + 1] - c->r[3 * j + 1], L[1]);
  double d2 = minimg(c->r[3 * i + 2] - c->r[3 * j + 2], L[2]);
  double dv = fma(d2, v[2], fma(d1, v[1], d0 * v[0]));
  *dv_out = dv;
  double dd = fma(d2, d2, fma(d1, d1, d0 * d0));
  double b2 = c->P.b_max * c->P.b_max;
  double rad = b2 - fma(-dv, dv, dd);
  if (rad < 0.0) rad = 0.0;
  double x = -dv + sqrt(rad);
  if (x < 0.0) x = 0.0;
  return x;
}

/* natural logarithm of u in (0, 1], an own routine from the textbook
 * reduction: u = m 2^e with m in [sqrt(1/2), sqrt(2)), log u = e ln 2 +
 * 2 atanh(z), z = (m - 1)/(m + 1) (|z| < 0.1716), atanh z / z =
 * sum_{n=0..14} z^(2n) / (2n + 1) by Horner's rule (the first term left out
 * is below 1e-19); ln 2 rounded to double.  Only +, -, *, / and exact bit
 * manipulations, so that another implementation taking the same steps gets
 * the same bits.  Within a few ulp of the correctly rounded value. */
double orc_log(double u) {
  uint64_t b;
  memcpy(&b, &u, sizeof(b));
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  const uint64_t mb = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
  double m;
  memcpy(&m, &mb, sizeof(m));
  if (m > 1.4142135623730951) {
    m = m * 0.5;
    e += 1;
  }
  const double z = (m - 1.0) / (m + 1.0);
  const double z2 = z * z;
  double s = 1.0 / 29.0;
  for (int n = 13; n >= 0; --n) s = s * z2 + 1.0 / (double)(2 * n + 1);
  return (double)e * 0.6931471805599453 + 2.0 * z * s;
}

/* Harmonic spring (k/2)(b - sigma)^2 between pivot i and its bonded bead j
 * (Sec. II, ECs with pair potentials): the pivot may move until the energy
 * its move adds reaches dE, drawn from the Boltzmann distribution.  Hard
 * spheres keep b >= sigma, so the energy falls while b falls and rises
 * only after the closest approach along the path (or from the start when
 * d.v >= 0): from the bond length b_s where it starts rising the pivot goes
 * on until b_t = sigma + sqrt((b_s - sigma)^2 + 2 dE / k), at
 * x = -d.v + sqrt(b_t^2 - |d_perp|^2). */
static double spring_x(double d0, double d1, double d2, const double v[3], double sigma, double k,
                       double dE, double *dv_out) {
  double dv = fma(d2, v[2], fma(d1, v[1], d0 * v[0]));
  *dv_out = dv;
  double dd = fma(d2, d2, fma(d1, d1, d0 * d0));
  double perp2 = fma(-dv, dv, dd);
  if (perp2 < 0.0) perp2 = 0.0;
  const double bs = dv < 0.0 ? sqrt(perp2) : sqrt(dd);
  const double e = bs - sigma;
  const double bt = sigma + sqrt(e * e + 2.0 * dE / k);
  /* b_t >= b_s >= |d_perp| exactly; rounding can leave the radicand a few
   * ulp below zero when dE ~ 0 and the path grazes the closest approach */
  double rad = bt * bt - perp2;
  if (rad < 0.0) rad = 0.0;
  double x = -dv + sqrt(rad);
  if (x < 0.0) x = 0.0;
  return x;
}

static double sp_dist(const ctx_t *c, int64_t i, int64_t j, const double v[3], double dE,
                      double *dv_out) {
  const double *L = c->P.L;
  double d0 = minimg(c->r[3 * i + 0] - c->r[3 * j + 0], L[0]);
  double d1 = minimg(c->r[3 * i + 1] - c->r[3 * j + 1], L[1]);
  double d2 = minimg(c->r[3 * i + 2] - c->r[3 * j + 2], L[2]);
  return spring_x(d0, d1, d2, v, c->P.sigma, c->P.k_spring, dE, dv_out);
}

/* the spring event of a pivot at separation d from its bonded bead, moving
 * along v with consumable energy dE (for the tests) */
double orc_spring_x(const double d[3], const double v[3], double sigma, double k, double dE) {
  double dv;
  return spring_x(d[0], d[1], d[2], v, sigma, k, dE, &dv);
}

static void hs_all(const ctx_t *c, int64_t i, const double v[3], cand_t *best) {
  if (c->P.use_cells) {
    int ci = c->cell[i];
    int ix = ci % c->nc[0];
    int iy = (ci / c->nc[0]) % c->nc[1];
    int iz = ci / (c->nc[0] * c->nc[1]);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int jx = (ix + dx + c->nc[0]) % c->nc[0];
          int jy = (iy + dy + c->nc[1]) % c->nc[1];
          int jz = (iz + dz + c->nc[2]) % c->nc[2];
          int cj = (jz * c->nc[1] + jy) * c->nc[0] + jx;
          for (int32_t k = c->head[cj]; k >= 0; k = c->next[k]) {
            if (k == i) continue;
            double dv;
            double x = hs_dist(c, i, k, v, &dv);
            if (x >= 0.0) consider(best, x, K_HS, k, dv);
          }
        }
  } else {
    for (int64_t k = 0; k < c->P.n; ++k) {
      if (k == i) continue;
      double dv;
      double x = hs_dist(c, i, k, v, &dv);
      if (x >= 0.0) consider(best, x, K_HS, k, dv);
    }
  }
}

/* ---------------------------------------------------------------------
 * one event chain
 * ------------------------------------------------------------------- */
typedef struct {
  int active;      /* domain mode */
  int32_t t;       /* tile index */
  double corner[3];
} tile_t;

static int motile(const ctx_t *c, const tile_t *tl, int64_t b) {
  return !tl->active || c->tag[b] == tl->t;
}

static void fnv(uint64_t *h, uint64_t w) {
  *h ^= w;
  *h *= 0x100000001B3ULL;
}

/* reflect v at the plane normal to d (Fig. 2c): v' = v - (2 v.d / d.d) d */
static void reflect(double v[3], double d0, double d1, double d2) {
  double dd = fma(d2, d2, fma(d1, d1, d0 * d0));
  double vd = fma(v[2], d2, fma(v[1], d1, v[0] * d0));
  double t = (2.0 * vd) / dd;
  v[0] = fma(-t, d0, v[0]);
  v[1] = fma(-t, d1, v[1]);
  v[2] = fma(-t, d2, v[2]);
}

/* swap test (Sec. II.C): with pivot i and the touched bead k exchanged,
 * every bond of i and of k must stay within b_max */
static int bond_ok(const ctx_t *c, int64_t a, const double *pa, int64_t b,
                   const double *pb) {
  const double *L = c->P.L;
  double d0 = minimg(pa[0] - pb[0], L[0]);
  double d1 = minimg(pa[1] - pb[1], L[1]);
  double d2 = minimg(pa[2] - pb[2], L[2]);
  double dd = fma(d2, d2, fma(d1, d1, d0 * d0));
  (void)a;
  (void)b;
  return dd <= c->P.b_max * c->P.b_max;
}

static const double *pos_after_swap(const ctx_t *c, int64_t q, int64_t i,
                                    int64_t k) {
  if (q == i) return &c->r[3 * k];
  if (q == k) return &c->r[3 * i];
  return &c->r[3 * q];
}

static int swap_allowed(const ctx_t *c, int64_t i, int64_t k) {
  int32_t N = c->P.N;
  int64_t ends[2] = {i, k};
  for (int e = 0; e < 2; ++e) {
    int64_t a = ends[e];
    int64_t nb[2] = {(a % N != 0) ? a - 1 : -1, (a % N != N - 1) ? a + 1 : -1};
    for (int s = 0; s < 2; ++s) {
      int64_t b = nb[s];
      if (b < 0) continue;
      if (!bond_ok(c, a, pos_after_swap(c, a, i, k), b,
                   pos_after_swap(c, b, i, k)))
        return 0;
    }
  }
  return 1;
}

static void exchange(ctx_t *c, int64_t i, int64_t k) {
  for (int a = 0; a < 3; ++a) {
    double tr = c->r[3 * i + a];
    c->r[3 * i + a] = c->r[3 * k + a];
    c->r[3 * k + a] = tr;
    int32_t ti = c->img[3 * i + a];
    c->img[3 * i + a] = c->img[3 * k + a];
    c->img[3 * k + a] = ti;
  }
  if (c->P.use_cells) {
    int ci = c->cell[i], ck = c->cell[k];
    if (ci != ck) {
      cell_remove(c, i);
      cell_remove(c, k);
      cell_insert(c, i, ck);
      cell_insert(c, k, ci);
    }
  }
}

static void run_ec(ctx_t *c, int64_t pivot, double v[3], double ell,
                   const tile_t *tl, uint64_t ec, uint64_t sweep,
                   uint64_t unit, int64_t ordinal) {
  const orc_params *P = &c->P;
  orc_stats *st = c->st;
  double xrem = ell;
  int64_t nev = 0, ncontact = 0;
  uint64_t h = 0xCBF29CE484222325ULL;
  double lift = 0.0;
  uint64_t sw[4] = {0, 0, 0, 0};
  for (;;) {
    if (nev >= P->event_cap) {
      st->status = ORC_ESTUCK;
      break;
    }
    const int64_t i = pivot;
    cand_t best = {xrem, K_END, -1, 0.0};
    consider(&best, P->s_cap, K_PASS, -1, 0.0);
    if (tl->active) {
      for (int a = 0; a < 3; ++a) {
        if (v[a] == 0.0) continue;
        double loc = minimg(c->r[3 * i + a] - tl->corner[a], P->L[a]);
        double x = (v[a] > 0.0) ? (c->W[a] - loc) / v[a] : (0.0 - loc) / v[a];
        if (x < 0.0) x = 0.0;
        consider(&best, x, K_WALL, a, 0.0);
      }
    }
    if (P->N > 1 && P->k_spring > 0.0) {
      /* springs: a fresh Boltzmann energy for each bond at every event,
       * dE = -log(u), u = 1 - u53 from Philox (tag 6 | ec << 8, sweep,
       * unit, event): word 0 for the bond to i - 1, word 1 for i + 1 */
      uint64_t w[4];
      draw(P, TAG_SPRING | (ec << 8), sweep, unit, (uint64_t)nev, w);
      double dv, x;
      if (i % P->N != 0) {
        x = sp_dist(c, i, i - 1, v, -orc_log(1.0 - u53(w[0])), &dv);
        consider(&best, x, K_TETHER, i - 1, dv);
      }
      if (i % P->N != P->N - 1) {
        x = sp_dist(c, i, i + 1, v, -orc_log(1.0 - u53(w[1])), &dv);
        consider(&best, x, K_TETHER, i + 1, dv);
      }
    } else if (P->N > 1) {
      double dv, x;
      if (i % P->N != 0) {
        x = te_dist(c, i, i - 1, v, &dv);
        consider(&best, x, K_TETHER, i - 1, dv);
      }
      if (i % P->N != P->N - 1) {
        x = te_dist(c, i, i + 1, v, &dv);
        consider(&best, x, K_TETHER, i + 1, dv);
      }
    }
    hs_all(c, i, v, &best);

    /* move the pivot */
    const double x = best.x;
    for (int a = 0; a < 3; ++a)
      advance(&c->r[3 * i + a], &c->img[3 * i + a], x, v[a], P->L[a]);
    cell_update(c, i);
    st->disp_sum += x;
    ++nev;
    ++st->events;

    int out;
    int64_t next = i;
    if (best.kind == K_END) {
      out = O_END;
    } else if (best.kind == K_PASS) {
      out = O_PASS;
    } else if (best.kind == K_WALL) {
      out = O_WALL;
      v[best.partner] = -v[best.partner];
    } else {
      const int64_t k = best.partner;
      double d0 = minimg(c->r[3 * i + 0] - c->r[3 * k + 0], P->L[0]);
      double d1 = minimg(c->r[3 * i + 1] - c->r[3 * k + 1], P->L[1]);
      double d2 = minimg(c->r[3 * i + 2] - c->r[3 * k + 2], P->L[2]);
      /* (r_k - r_i).v at contact = -(d.v) - x, d the separation before the
       * flight x (the pressure projection, R8) */
      double proj = -best.dv - x;
      if (!motile(c, tl, k)) {
        /* partner cannot move: reflect at the contact / bond normal */
        out = (best.kind == K_HS) ? O_HS_REFLECT : O_TE_REFLECT;
        st->refl_sum += proj;
        reflect(v, d0, d1, d2);
      } else if (best.kind == K_HS) {
        lift += proj;
        int swapped = 0;
        if (P->p_swap > 0.0) {
          int go;
          if (P->p_swap >= 1.0) {
            go = 1;
          } else {
            if ((ncontact & 3) == 0)
              draw(P, TAG_SWAP | (ec << 8), sweep, unit, (uint64_t)(ncontact >> 2), sw);
            go = u53(sw[ncontact & 3]) < P->p_swap;
          }
          ++ncontact;
          if (go) {
            ++st->swap_tried;
            if (swap_allowed(c, i, k)) {
              exchange(c, i, k);
              swapped = 1;
            }
          }
        }
        if (swapped) {
          out = O_SWAP;
        } else {
          out = O_HS_LIFT;
          next = k;
        }
      } else {
        lift += proj;
        out = O_TE_LIFT;
        next = k;
      }
    }
    st->out[out] += 1;
    fnv(&h, (uint64_t)i);
    fnv(&h, ((uint64_t)(uint32_t)out << 32) | (uint64_t)(uint32_t)best.partner);
    {
      uint64_t xb;
      memcpy(&xb, &x, 8);
      fnv(&h, xb);
    }
    if (c->log && *c->log_n < c->log_cap) {
      orc_event *e = &c->log[*c->log_n];
      e->unit = ordinal;
      e->pivot = (int32_t)i;
      e->kind = out;
      e->partner = best.partner;
      e->x = x;
      *c->log_n += 1;
    }
    if (out == O_END) break;
    xrem = xrem - x;
    pivot = next;
  }
  st->lift_sum += lift;
  st->ecs += 1;
  if (ordinal >= 0) {
    if (c->digest) c->digest[ordinal] = h;
    if (c->ec_lift) c->ec_lift[ordinal] = lift;
    if (c->ec_events) c->ec_events[ordinal] = nev;
  }
}

/* direction: {+x,+y,+z} (global balance, Sec. II), isotropic by rejection
 * from the cube (no trigonometry), or +x only (one-dimensional checks) */
static void draw_start(const ctx_t *c, uint64_t tag, uint64_t sweep,
                       uint64_t unit, int64_t m, int64_t *idx, double v[3]) {
  uint64_t w[4];
  draw(&c->P, tag, sweep, unit, 0, w);
  *idx = below(w[0], m);
  v[0] = v[1] = v[2] = 0.0;
  if (c->P.dir_mode == ORC_DIR_CART3) {
    v[below(w[1], 3)] = 1.0;
  } else if (c->P.dir_mode == ORC_DIR_PLUSX) {
    v[0] = 1.0;
  } else {
    uint64_t a = 0;
    double p = 2.0 * u53(w[1]) - 1.0;
    double q = 2.0 * u53(w[2]) - 1.0;
    double s3 = 2.0 * u53(w[3]) - 1.0;
    for (;;) {
      double s = p * p + q * q + s3 * s3;
      if (s > 1e-6 && s <= 1.0) {
        double nr = sqrt(s);
        v[0] = p / nr;
        v[1] = q / nr;
        v[2] = s3 / nr;
        break;
      }
      ++a;
      draw(&c->P, tag, sweep, unit, a, w);
      p = 2.0 * u53(w[0]) - 1.0;
      q = 2.0 * u53(w[1]) - 1.0;
      s3 = 2.0 * u53(w[2]) - 1.0;
    }
  }
}

/* ---------------------------------------------------------------------
 * public entry points (ctypes)
 * ------------------------------------------------------------------- */

/* serial, undecomposed: EC j (j = 0..n_ec-1 of this call, global ordinal
 * ec0 + j) starts at a uniform bead with a direction from Philox. */
int orc_run_serial(const orc_params *P, double *r, int32_t *img, int64_t ec0,
                   int64_t n_ec, double ell, orc_stats *st, uint64_t *digest,
                   double *ec_lift, int64_t *ec_events, orc_event *log,
                   int64_t log_cap, int64_t *log_n) {
  if (P->n < 1 || P->N < 1 || P->n % P->N != 0 || !(P->sigma > 0.0) ||
      !(P->s_cap > 0.0) || !(ell >= 0.0))
    return ORC_EINVAL;
  if (!(P->k_spring >= 0.0) || (P->k_spring > 0.0 && P->p_swap > 0.0)) return ORC_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!(P->s_cap + P->sigma < 0.5 * P->L[a])) return ORC_EINVAL;
  ctx_t c;
  ctx_init(&c, P, r, img);
  c.st = st;
  c.log = log;
  c.log_cap = log_cap;
  c.log_n = log_n;
  c.digest = digest;
  c.ec_lift = ec_lift;
  c.ec_events = ec_events;
  tile_t tl = {0, 0, {0, 0, 0}};
  for (int64_t j = 0; j < n_ec && st->status == 0; ++j) {
    int64_t idx;
    double v[3];
    draw_start(&c, TAG_START, 0, (uint64_t)(ec0 + j), P->n, &idx, v);
    run_ec(&c, idx, v, ell, &tl, 0, 0, (uint64_t)(ec0 + j), j);
  }
  ctx_free(&c);
  return (int)st->status;
}

/* domain assignment (Sec. II.A): shift o in [0,T)^3 drawn per sweep; along
 * each axis tile k covers [o + kT, o + (k+1)T - w), the last w is joint. */
static void domain_setup(ctx_t *c, uint64_t sweep) {
  const orc_params *P = &c->P;
  uint64_t w[4];
  draw(P, TAG_SHIFT, sweep, 0, 0, w);
  for (int a = 0; a < 3; ++a) {
    c->T[a] = P->L[a] / P->D[a];
    c->W[a] = c->T[a] - P->w;
    c->shift[a] = u53(w[a]) * c->T[a];
  }
  for (int64_t b = 0; b < P->n; ++b) {
    int k[3], in = 1;
    for (int a = 0; a < 3; ++a) {
      double u = c->r[3 * b + a] - c->shift[a];
      if (u < 0.0) u += P->L[a];
      if (u >= P->L[a]) u -= P->L[a];
      int t = (int)(u / c->T[a]);
      if (t > P->D[a] - 1) t = P->D[a] - 1;
      double loc = u - t * c->T[a];
      if (!(loc < c->W[a])) in = 0;
      k[a] = t;
    }
    c->tag[b] = in ? (k[2] * P->D[1] + k[1]) * P->D[0] + k[0] : -1;
  }
  if (P->k_spring > 0.0 && P->N > 1) {
    /* springs have no longest bond: a bead whose bonded bead is motile in
     * another tile would couple the two tiles, so both wait (reading R23);
     * decided on the tags above, then applied */
    int8_t *drop = (int8_t *)calloc((size_t)P->n, 1);
    for (int64_t b = 0; b < P->n; ++b) {
      if (c->tag[b] < 0) continue;
      const int64_t nb[2] = {b % P->N != 0 ? b - 1 : -1, b % P->N != P->N - 1 ? b + 1 : -1};
      for (int q = 0; q < 2; ++q)
        if (nb[q] >= 0 && c->tag[nb[q]] >= 0 && c->tag[nb[q]] != c->tag[b]) drop[b] = 1;
    }
    for (int64_t b = 0; b < P->n; ++b)
      if (drop[b]) c->tag[b] = -1;
    free(drop);
  }
}

int orc_domain_tags(const orc_params *P, double *r, uint64_t sweep,
                    int32_t *tags_out, double *shift_out) {
  int32_t dummy_img[3] = {0, 0, 0};
  orc_params Q = *P;
  Q.use_cells = 0;
  ctx_t c;
  ctx_init(&c, &Q, r, dummy_img);
  domain_setup(&c, sweep);
  memcpy(tags_out, c.tag, sizeof(int32_t) * P->n);
  for (int a = 0; a < 3; ++a) shift_out[a] = c.shift[a];
  ctx_free(&c);
  return 0;
}

/* domain-parallel sweeps: tiles are independent within a sweep (joint width
 * w >= b_max > sigma), so running them one after another in increasing tile
 * index gives the same result as running them at the same time. */
int orc_run_domain(const orc_params *P, double *r, int32_t *img, int64_t sweep0,
                   int64_t n_sweeps, double ell, orc_stats *st,
                   uint64_t *digest, double *ec_lift, int64_t *ec_events,
                   orc_event *log, int64_t log_cap, int64_t *log_n) {
  if (P->n < 1 || P->N < 1 || P->n % P->N != 0 || !(P->sigma > 0.0) ||
      !(P->s_cap > 0.0) || !(ell >= 0.0) || P->ecs_per_tile < 1)
    return ORC_EINVAL;
  if (!(P->w >= P->b_max) || !(P->b_max >= P->sigma)) return ORC_EINVAL;
  if (!(P->k_spring >= 0.0) || (P->k_spring > 0.0 && P->p_swap > 0.0)) return ORC_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (P->D[a] < 1) return ORC_EINVAL;
    double T = P->L[a] / P->D[a];
    if (!(T - P->w + 2.0 * P->sigma < 0.5 * P->L[a])) return ORC_EINVAL;
    if (!(P->s_cap + P->sigma < 0.5 * P->L[a])) return ORC_EINVAL;
  }
  ctx_t c;
  ctx_init(&c, P, r, img);
  c.st = st;
  c.log = log;
  c.log_cap = log_cap;
  c.log_n = log_n;
  c.digest = digest;
  c.ec_lift = ec_lift;
  c.ec_events = ec_events;
  const int64_t ntile = (int64_t)P->D[0] * P->D[1] * P->D[2];
  const int k = P->ecs_per_tile;
  int64_t *cnt = (int64_t *)calloc(ntile + 1, sizeof(int64_t));
  int64_t *list = (int64_t *)malloc(sizeof(int64_t) * P->n);
  for (int64_t s = 0; s < n_sweeps && st->status == 0; ++s) {
    const uint64_t sweep = (uint64_t)(sweep0 + s);
    domain_setup(&c, sweep);
    /* motile beads of every tile, in increasing bead id */
    memset(cnt, 0, sizeof(int64_t) * (ntile + 1));
    for (int64_t b = 0; b < P->n; ++b)
      if (c.tag[b] >= 0) cnt[c.tag[b] + 1] += 1;
    for (int64_t t = 0; t < ntile; ++t) cnt[t + 1] += cnt[t];
    {
      int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (ntile + 1));
      memcpy(fill, cnt, sizeof(int64_t) * (ntile + 1));
      for (int64_t b = 0; b < P->n; ++b)
        if (c.tag[b] >= 0) list[fill[c.tag[b]]++] = b;
      free(fill);
    }
    for (int64_t t = 0; t < ntile && st->status == 0; ++t) {
      if (P->tile_mod > 1 && t % P->tile_mod != P->tile_rem) continue;
      int64_t m = cnt[t + 1] - cnt[t];
      if (m == 0) continue;
      tile_t tl;
      tl.active = 1;
      tl.t = (int32_t)t;
      int kx = (int)(t % P->D[0]);
      int ky = (int)((t / P->D[0]) % P->D[1]);
      int kz = (int)(t / ((int64_t)P->D[0] * P->D[1]));
      tl.corner[0] = c.shift[0] + kx * c.T[0];
      tl.corner[1] = c.shift[1] + ky * c.T[1];
      tl.corner[2] = c.shift[2] + kz * c.T[2];
      if (P->pushoff) {
        /* one EC from every flagged motile bead, in bead id order; the
         * direction is EC e's usual draw */
        int e = 0;
        for (int64_t q = cnt[t]; q < cnt[t + 1] && st->status == 0; ++q) {
          if (!P->po_flag[list[q]]) continue;
          int64_t idx;
          double v[3];
          draw_start(&c, TAG_START | ((uint64_t)e << 8), sweep, (uint64_t)t, m, &idx, v);
          run_ec(&c, list[q], v, ell, &tl, (uint64_t)e, sweep, (uint64_t)t, -1);
          ++e;
        }
        continue;
      }
      for (int e = 0; e < k && st->status == 0; ++e) {
        int64_t idx;
        double v[3];
        draw_start(&c, TAG_START | ((uint64_t)e << 8), sweep, (uint64_t)t, m,
                   &idx, v);
        int64_t ord = (s * ntile + t) * k + e;
        run_ec(&c, list[cnt[t] + idx], v, ell, &tl, (uint64_t)e, sweep,
               (uint64_t)t, ord);
      }
    }
  }
  free(cnt);
  free(list);
  ctx_free(&c);
  return (int)st->status;
}

/* ---------------------------------------------------------------------
 * initial state and observables
 * ------------------------------------------------------------------- */

/* simple-cubic lattice n0 x n1 x n2 with spacing a, visited in a 3-D snake
 * (x fastest and reversing every row, y reversing every plane), cut into
 * consecutive runs of N = chains.  Every bond is one lattice step.  Each
 * coordinate is then moved by jitter*(2u-1), u from Philox (tag 4, unit =
 * bead): an exact lattice combined with {+x,+y,+z} directions holds bonded
 * pairs with equal coordinates whose bond, once taut and perpendicular to v,
 * stops the hard-tether EC (zero-length tether events back and forth). */
int orc_lattice(const int32_t dims[3], double a, double jitter, uint64_t seed,
                uint64_t replica, double *r) {
  orc_params P;
  memset(&P, 0, sizeof(P));
  P.seed = seed;
  P.replica = replica;
  int64_t b = 0;
  for (int z = 0; z < dims[2]; ++z) {
    for (int yy = 0; yy < dims[1]; ++yy) {
      int y = (z % 2 == 0) ? yy : dims[1] - 1 - yy;
      int row = z * dims[1] + yy;
      for (int xx = 0; xx < dims[0]; ++xx) {
        int x = (row % 2 == 0) ? xx : dims[0] - 1 - xx;
        int site[3] = {x, y, z};
        uint64_t w[4] = {0, 0, 0, 0};
        if (jitter != 0.0) draw(&P, 4, 0, (uint64_t)b, 0, w);
        for (int ax = 0; ax < 3; ++ax) {
          double p = (site[ax] + 0.5) * a;
          if (jitter != 0.0) p = p + jitter * (2.0 * u53(w[ax]) - 1.0);
          r[3 * b + ax] = p;
        }
        ++b;
      }
    }
  }
  return 0;
}

/* per-chain end-to-end vector from minimum-image bonds, per-bond lengths */
int orc_chain_obs(const orc_params *P, const double *r, double *re2_chain,
                  double *bond_len) {
  int64_t nch = P->n / P->N;
  for (int64_t ch = 0; ch < nch; ++ch) {
    double R[3] = {0, 0, 0};
    for (int32_t j = 0; j + 1 < P->N; ++j) {
      int64_t b = ch * P->N + j;
      double dd = 0.0;
      for (int a = 0; a < 3; ++a) {
        double d = minimg(r[3 * (b + 1) + a] - r[3 * b + a], P->L[a]);
        R[a] += d;
        dd += d * d;
      }
      if (bond_len) bond_len[ch * (P->N - 1) + j] = sqrt(dd);
    }
    re2_chain[ch] = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  }
  return 0;
}

/* smallest pair distance (all pairs, minimum image) and the number of pairs
 * closer than sigma*(1 - 1e-10)^(1/2) */
int orc_min_pair(const orc_params *P, const double *r, double *dmin,
                 int64_t *n_overlap) {
  double best = INFINITY;
  int64_t cnt = 0;
  double lim = P->sigma * P->sigma * (1.0 - 1e-10);
  for (int64_t i = 0; i < P->n; ++i)
    for (int64_t j = i + 1; j < P->n; ++j) {
      double dd = 0.0;
      for (int a = 0; a < 3; ++a) {
        double d = minimg(r[3 * i + a] - r[3 * j + a], P->L[a]);
        dd += d * d;
      }
      if (dd < best) best = dd;
      if (dd < lim) ++cnt;
    }
  *dmin = sqrt(best);
  *n_overlap = cnt;
  return 0;
}

/* same check through the oracle's own cell list (large systems) */
int orc_min_pair_cells(const orc_params *P, double *r, double *dmin,
                       int64_t *n_overlap) {
  orc_params Q = *P;
  Q.use_cells = 1;
  Q.s_cap = 0.25 * P->sigma;
  int32_t dummy[3] = {0, 0, 0};
  ctx_t c;
  ctx_init(&c, &Q, r, dummy);
  if (!c.P.use_cells) {
    ctx_free(&c);
    return orc_min_pair(P, r, dmin, n_overlap);
  }
  double best = INFINITY;
  int64_t cnt = 0;
  double lim = P->sigma * P->sigma * (1.0 - 1e-10);
  for (int64_t i = 0; i < P->n; ++i) {
    int ci = c.cell[i];
    int ix = ci % c.nc[0], iy = (ci / c.nc[0]) % c.nc[1],
        iz = ci / (c.nc[0] * c.nc[1]);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int cj = (((iz + dz + c.nc[2]) % c.nc[2]) * c.nc[1] +
                    (iy + dy + c.nc[1]) % c.nc[1]) * c.nc[0] +
                   (ix + dx + c.nc[0]) % c.nc[0];
          for (int32_t j = c.head[cj]; j >= 0; j = c.next[j]) {
            if (j <= i) continue;
            double dd = 0.0;
            for (int a = 0; a < 3; ++a) {
              double d = minimg(r[3 * i + a] - r[3 * j + a], P->L[a]);
              dd += d * d;
            }
            if (dd < best) best = dd;
            if (dd < lim) ++cnt;
          }
        }
  }
  ctx_free(&c);
  *dmin = sqrt(best);
  *n_overlap = cnt;
  return 0;
}

/* Contact counts behind the configurational pressure (the virial theorem
 * for hard constraints): pairs with |r_ij| in [sigma, sigma + delta) and
 * [sigma + delta, sigma + 2 delta) (the first shell also takes pairs a
 * rounding error inside sigma, as the overlap test does), and bonds with
 * length in (b_max - delta, b_max] and (b_max - 2 delta, b_max - delta]
 * (the first shell up to the tether-violation tolerance).  Brute force over
 * every pair. */
int orc_contacts(const orc_params *P, const double *r, double delta, int64_t *pairs,
                 int64_t *bonds) {
  const double lo = P->sigma * P->sigma * (1.0 - 1e-10);
  const double s1 = (P->sigma + delta) * (P->sigma + delta);
  const double s2 = (P->sigma + 2.0 * delta) * (P->sigma + 2.0 * delta);
  const double t0 = P->b_max * P->b_max * (1.0 + 1e-10);
  const double t1 = (P->b_max - delta) * (P->b_max - delta);
  const double t2 = (P->b_max - 2.0 * delta) * (P->b_max - 2.0 * delta);
  pairs[0] = pairs[1] = 0;
  bonds[0] = bonds[1] = 0;
  for (int64_t i = 0; i < P->n; ++i)
    for (int64_t j = i + 1; j < P->n; ++j) {
      double dd = 0.0;
      for (int a = 0; a < 3; ++a) {
        double d = minimg(r[3 * i + a] - r[3 * j + a], P->L[a]);
        dd += d * d;
      }
      if (dd >= lo && dd < s1) ++pairs[0];
      else if (dd >= s1 && dd < s2) ++pairs[1];
    }
  for (int64_t b = 0; b + 1 < P->n; ++b) {
    if ((b + 1) % P->N == 0) continue; /* b is the last bead of its chain */
    double dd = 0.0;
    for (int a = 0; a < 3; ++a) {
      double d = minimg(r[3 * (b + 1) + a] - r[3 * b + a], P->L[a]);
      dd += d * d;
    }
    if (dd > t1 && dd <= t0) ++bonds[0];
    else if (dd > t2 && dd <= t1) ++bonds[1];
  }
  return 0;
}

/* start draws of serial ECs ec0..ec0+n-1 (for the direction/start checks) */
int orc_start_draws(const orc_params *P, int64_t ec0, int64_t n, int64_t *idx,
                    double *v) {
  ctx_t c;
  memset(&c, 0, sizeof(c));
  c.P = *P;
  for (int64_t j = 0; j < n; ++j)
    draw_start(&c, TAG_START, 0, (uint64_t)(ec0 + j), P->n, &idx[j], &v[3 * j]);
  return 0;
}

/*
 * Chain structure of the current state, each quantity written out from its
 * definition:
 *   - radius of gyration R_g^2 and the centre of mass R (Sec. IV, the
 *     plateau of g2), and the moment of inertia tensor of a chain (Appendix
 *     A), through the gyration tensor S = (1/N) sum_j (u_j - U)(u_j - U)^T
 *     with U = (1/N) sum_j u_j (the inertia tensor is N (Tr S 1 - S));
 *   - the middle bead relative to the centre of mass, u_{N/2} - U (the
 *     quantity whose displacement g2 averages, Sec. IV);
 *   - mean-square internal distances R^2(n) (Sec. II.B):
 *     r2n[n] = mean over chains and j of |u_{j+n} - u_j|^2, r2n[0] = 0;
 *   - the end-to-end distance distribution W(R) (Appendix A) as counts of
 *     chains with floor(|u_{N-1} - u_0| / dR) = b, the last bin taking the
 *     rest.
 * u_j are the positions along a chain from minimum-image bonds:
 * u_0 = 0, u_{j+1} = u_j + minimg(r_{j+1} - r_j).  Sums run in index order
 * (beads, then chains); any output may be NULL.
 *   gyr[6 ch + k]: S_xx, S_xy, S_xz, S_yy, S_yz, S_zz
 *   mid[3 ch + a]: u_{N/2} - U
 */
int orc_chain_struct(const orc_params *P, const double *r, double *gyr, double *mid,
                     double *r2n, double dR, int64_t nbins, int64_t *hist) {
  const int32_t N = P->N;
  const int64_t nch = P->n / N;
  double *u = (double *)malloc(sizeof(double) * 3 * (size_t)N);
  double *acc = r2n ? (double *)calloc((size_t)N, sizeof(double)) : NULL;
  if (!u || (r2n && !acc)) {
    free(u);
    free(acc);
    return ORC_EINVAL;
  }
  if (hist)
    for (int64_t b = 0; b < nbins; ++b) hist[b] = 0;
  for (int64_t ch = 0; ch < nch; ++ch) {
    const double *rc = r + 3 * ch * N;
    u[0] = u[1] = u[2] = 0.0;
    for (int32_t j = 0; j + 1 < N; ++j)
      for (int a = 0; a < 3; ++a)
        u[3 * (j + 1) + a] = u[3 * j + a] + minimg(rc[3 * (j + 1) + a] - rc[3 * j + a], P->L[a]);
    double U[3];
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int32_t j = 0; j < N; ++j) s += u[3 * j + a];
      U[a] = s / (double)N;
    }
    if (gyr) {
      double s00 = 0.0, s01 = 0.0, s02 = 0.0, s11 = 0.0, s12 = 0.0, s22 = 0.0;
      for (int32_t j = 0; j < N; ++j) {
        const double d0 = u[3 * j] - U[0], d1 = u[3 * j + 1] - U[1], d2 = u[3 * j + 2] - U[2];
        s00 += d0 * d0;
        s01 += d0 * d1;
        s02 += d0 * d2;
        s11 += d1 * d1;
        s12 += d1 * d2;
        s22 += d2 * d2;
      }
      double *g = gyr + 6 * ch;
      g[0] = s00 / (double)N;
      g[1] = s01 / (double)N;
      g[2] = s02 / (double)N;
      g[3] = s11 / (double)N;
      g[4] = s12 / (double)N;
      g[5] = s22 / (double)N;
    }
    if (mid)
      for (int a = 0; a < 3; ++a) mid[3 * ch + a] = u[3 * (N / 2) + a] - U[a];
    if (hist && nbins > 0) {
      const double *e = u + 3 * (N - 1);
      const double R = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
      int64_t b = (int64_t)floor(R / dR);
      if (b >= nbins) b = nbins - 1;
      ++hist[b];
    }
    if (acc)
      for (int32_t n = 1; n < N; ++n) {
        double part = 0.0;
        for (int32_t j = 0; j + n < N; ++j) {
          const double d0 = u[3 * (j + n)] - u[3 * j];
          const double d1 = u[3 * (j + n) + 1] - u[3 * j + 1];
          const double d2 = u[3 * (j + n) + 2] - u[3 * j + 2];
          part += d0 * d0 + d1 * d1 + d2 * d2;
        }
        acc[n] += part;
      }
  }
  if (r2n) {
    r2n[0] = 0.0;
    for (int32_t n = 1; n < N; ++n) r2n[n] = acc[n] / ((double)nch * (double)(N - n));
  }
  free(u);
  free(acc);
  return 0;
}

/*
 * Phantom chains for the initial configuration (Sec. II.B, first stage of
 * the slow push-off): n_chains chains of N beads without excluded volume,
 * each a non-reversal random walk with bond length `bond`.  The first bead
 * is uniform in the box, the first bond uniform on the sphere, and every
 * next bond t_{j+1} uniform on the cap t_j . t_{j+1} >= ct around the one
 * before, ct = cos(theta_max) = (c - 3)/(c + 1): then <cos theta> =
 * (1 + ct)/2 = cos^2(theta_max/2) = (c - 1)/(c + 1) and
 * <R^2> -> c (N - 1) bond^2 for long chains, c the paper's stiffness
 * parameter.  (The paper writes the cap with "<"; its own <cos theta>
 * holds for ">=", reading R21.)
 * Random numbers: Philox4x64-10, key (seed, 0), counter (5, chain, bead,
 * attempt).  Bead 0: words 0-2 times L.  Bead j >= 1: cos theta =
 * 1 - u(w0) (1 - ct_j) (ct_1 = -1: the whole sphere); the azimuth from the
 * first point (x, y) = (2 u - 1, 2 u' - 1) with 0 < x^2 + y^2 <= 1, taken
 * from words 1, 2 of attempt 0, then words 0, 1 of attempts 1, 2, ...
 * (at most 256 attempts, else an error);
 * t_{j+1} = cos theta t_j + sin theta (cos phi e1 + sin phi e2) with the
 * orthonormal pair (e1, e2) of t_j from Duff et al., "Building an
 * orthonormal basis, revisited" (JCGT 6(1), 2017), then normalised; the
 * tangent before bond 1 is e_z.  Positions are then wrapped as the library
 * wraps caller input: f = floor(x / L), x -= f L, x >= L -> x - L,
 * x < 0 -> 0, image f.
 */
int orc_phantom(const double L[3], int64_t nch, int32_t N, double bond, double c, uint64_t seed,
                double *r, int32_t *img) {
  const double ct = (c - 3.0) / (c + 1.0);
  const uint64_t key[2] = {seed, 0};
  for (int64_t ch = 0; ch < nch; ++ch) {
    uint64_t ctr[4] = {5, (uint64_t)ch, 0, 0}, w[4];
    orc_philox4x64_10(ctr, key, w);
    double p[3], t[3] = {0.0, 0.0, 1.0};
    for (int a = 0; a < 3; ++a) p[a] = u53(w[a]) * L[a];
    double *rc = r + 3 * ch * N;
    for (int a = 0; a < 3; ++a) rc[a] = p[a];
    for (int32_t j = 1; j < N; ++j) {
      const double ctj = j == 1 ? -1.0 : ct;
      uint64_t cj[4] = {5, (uint64_t)ch, (uint64_t)j, 0};
      orc_philox4x64_10(cj, key, w);
      const double cth = 1.0 - u53(w[0]) * (1.0 - ctj);
      double x = 2.0 * u53(w[1]) - 1.0, y = 2.0 * u53(w[2]) - 1.0;
      double s = x * x + y * y;
      for (uint64_t att = 1; !(s > 0.0 && s <= 1.0); ++att) {
        if (att == 256) return ORC_EINVAL; /* (probability 0.21^256) */
        cj[3] = att;
        orc_philox4x64_10(cj, key, w);
        x = 2.0 * u53(w[0]) - 1.0;
        y = 2.0 * u53(w[1]) - 1.0;
        s = x * x + y * y;
      }
      const double sq = sqrt(s);
      const double cph = x / sq, sph = y / sq;
      const double sth = sqrt(1.0 - cth * cth);
      const double sg = t[2] >= 0.0 ? 1.0 : -1.0;
      const double aa = -1.0 / (sg + t[2]);
      const double bb = t[0] * t[1] * aa;
      const double e1[3] = {1.0 + sg * t[0] * t[0] * aa, sg * bb, -sg * t[0]};
      const double e2[3] = {bb, sg + t[1] * t[1] * aa, -t[1]};
      double nt[3];
      for (int a = 0; a < 3; ++a) nt[a] = cth * t[a] + sth * (cph * e1[a] + sph * e2[a]);
      const double q = sqrt(nt[0] * nt[0] + nt[1] * nt[1] + nt[2] * nt[2]);
      for (int a = 0; a < 3; ++a) {
        t[a] = nt[a] / q;
        p[a] = p[a] + bond * t[a];
        rc[3 * j + a] = p[a];
      }
    }
  }
  for (int64_t i = 0; i < 3 * nch * N; ++i) {
    const double La = L[i % 3];
    double x = r[i];
    const double f = floor(x / La);
    x -= f * La;
    if (x >= La) x -= La;
    if (x < 0) x = 0;
    r[i] = x;
    img[i] = (int32_t)f;
  }
  return 0;
}

/*
 * Beads that overlap another bead at diameter d: |r_i - r_k|^2 <
 * d^2 (1 - 1e-10), minimum image, squared length summed as
 * d0 d0 + d1 d1 + d2 d2.  A grid of cells no narrower than d (all pairs
 * when an axis has fewer than three cells).  flag[i] = 1 or 0; returns the
 * number flagged.
 */
int64_t orc_overlap_flags(const orc_params *P, const double *r, double d, uint8_t *flag) {
  const double thr = d * d * (1.0 - 1e-10);
  int nc[3];
  int cells = 1;
  for (int a = 0; a < 3; ++a) {
    nc[a] = (int)floor(P->L[a] / d);
    if (nc[a] > 256) nc[a] = 256;
    if (nc[a] < 3) cells = 0;
  }
  for (int64_t i = 0; i < P->n; ++i) flag[i] = 0;
  if (!cells) {
    for (int64_t i = 0; i < P->n; ++i)
      for (int64_t k = i + 1; k < P->n; ++k) {
        double dd = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double x = minimg(r[3 * i + a] - r[3 * k + a], P->L[a]);
          dd += x * x;
        }
        if (dd < thr) flag[i] = flag[k] = 1;
      }
  } else {
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)P->n);
    int64_t *cellof = (int64_t *)malloc(sizeof(int64_t) * (size_t)P->n);
    for (int64_t i = 0; i < P->n; ++i) {
      int64_t ci = 0;
      for (int a = 2; a >= 0; --a) {
        int x = (int)floor(r[3 * i + a] / (P->L[a] / nc[a]));
        if (x < 0) x = 0;
        if (x >= nc[a]) x = nc[a] - 1;
        ci = ci * nc[a] + x;
      }
      cellof[i] = ci;
      start[ci + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    {
      int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
      memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
      for (int64_t i = 0; i < P->n; ++i) order[fill[cellof[i]]++] = i;
      free(fill);
    }
    for (int64_t i = 0; i < P->n; ++i) {
      const int64_t ci = cellof[i];
      const int cx = (int)(ci % nc[0]), cy = (int)((ci / nc[0]) % nc[1]), cz = (int)(ci / ((int64_t)nc[0] * nc[1]));
      for (int dz = -1; dz <= 1 && !flag[i]; ++dz)
        for (int dy = -1; dy <= 1 && !flag[i]; ++dy)
          for (int dx = -1; dx <= 1 && !flag[i]; ++dx) {
            const int x = (cx + dx + nc[0]) % nc[0], y = (cy + dy + nc[1]) % nc[1], z = (cz + dz + nc[2]) % nc[2];
            const int64_t cj = ((int64_t)z * nc[1] + y) * nc[0] + x;
            for (int64_t q = start[cj]; q < start[cj + 1]; ++q) {
              const int64_t k = order[q];
              if (k == i) continue;
              double dd = 0.0;
              for (int a = 0; a < 3; ++a) {
                const double y2 = minimg(r[3 * i + a] - r[3 * k + a], P->L[a]);
                dd += y2 * y2;
              }
              if (dd < thr) {
                flag[i] = 1;
                break;
              }
            }
          }
    }
    free(start);
    free(order);
    free(cellof);
  }
  int64_t m = 0;
  for (int64_t i = 0; i < P->n; ++i) m += flag[i];
  return m;
}

/*
 * Slow push-off (Sec. II.B): from chains that may overlap (phantom chains),
 * grow the hard-sphere diameter from f0 sigma to sigma in `stages` equal
 * steps, d_k = sigma (f0 + (1 - f0) k / stages) and d_stages = sigma; at
 * every diameter, repeat domain sweeps (tiles and shifts as in the EC run,
 * swaps off) whose ECs start at the beads that overlap, one EC each, and
 * whose pivot ignores the beads it overlaps, until no overlap is left.
 * Sweeps are numbered from sweep0; *sweeps_out receives their number.
 * ORC_ESTUCK when a diameter is not resolved within max_sweeps sweeps.
 */
int orc_pushoff(const orc_params *P0, double *r, int32_t *img, double f0, int32_t stages,
                double ell, int64_t max_sweeps, int64_t sweep0, int64_t *sweeps_out,
                orc_stats *st) {
  if (!(f0 > 0.0 && f0 <= 1.0) || stages < 1 || max_sweeps < 1) return ORC_EINVAL;
  orc_params P = *P0;
  P.mode = ORC_DOMAIN;
  P.pushoff = 1;
  P.p_swap = 0.0;
  uint8_t *flag = (uint8_t *)malloc((size_t)P.n);
  P.po_flag = flag;
  int64_t sweeps = 0;
  int rc = 0;
  for (int32_t k = 0; k <= stages && rc == 0; ++k) {
    const double d = k == stages ? P0->sigma : P0->sigma * (f0 + (1.0 - f0) * (double)k / (double)stages);
    P.sigma = d;
    for (int64_t s = 0;; ++s) {
      if (orc_overlap_flags(&P, r, d, flag) == 0) break;
      if (s == max_sweeps) {
        rc = ORC_ESTUCK;
        break;
      }
      rc = orc_run_domain(&P, r, img, sweep0 + sweeps, 1, ell, st, NULL, NULL, NULL, NULL, 0, NULL);
      ++sweeps;
      if (rc) break;
    }
  }
  free(flag);
  *sweeps_out = sweeps;
  return rc;
}
