// Block-lockstep EC kernel of the screened domain form (arXiv:1502.06447,
// Sec. II: EC move with hard tethers; Sec. II.A: tiles, joints and
// reflections; Sec. II.C: swap move).  Bead springs run in the warp-lockstep
// kernel (k_ec.cu).
//
// A block runs NT tiles.  Each tile is staged and screened by a group of G
// lanes exactly as in ec_kernel, but all NT tiles advance one event per step
// in lockstep and the FP64 work of the step is packed one tile per lane:
//   A  every group bounds its pivot's candidates in FP32 (contacts in the 27
//      local cells, tethers, tile walls) and appends each candidate whose
//      lower bound can reach the smallest upper bound U to the block's
//      request list;
//   B  the requests of all tiles are evaluated in FP64, one per thread;
//   D  thread t (t < NT) picks tile t's winner among its evaluated requests
//      and the END/PASS candidate, moves the pivot, lifts, reflects or swaps,
//      and sets up the next step (or the tile's next EC).
// An FP64 warp instruction costs the same whatever its active mask, so
// phases B and D serve up to 32 tiles per FP64 instruction where the G-lane
// groups of ec_kernel serve 32/G.  Every event is the one ec_kernel (and the
// oracle) produces: same candidates, same FP64 expressions, same tie rule.
// A tile whose survivors do not fit the request list (rare) is evaluated
// exhaustively in FP64 by its own group in phase B.
//
// FP64 positions stay in the global array (the owner thread updates its
// pivot's in place; no other tile touches those beads), so shared memory
// holds only the FP32 shadows, ids, bond words and local grid of each tile;
// an evaluated request carries its partner's position to phase D.
#include <type_traits>

#include "ec_device.cuh"

namespace ecmc {
namespace {

// per-tile record shared by the group (A), the evaluating threads (B) and
// the owner thread (D)
struct __align__(16) TileRec {
  double q[3], v[3];  // pivot position (wrapped FP64) and direction
  double c[3];        // tile corner
  float pf[3], vf[3];
  float xcap;         // FP32 upper bound of the END/PASS candidate
  int p;              // pivot slot
  int active;
  int vnz;            // bit a: v_a != 0
  int rq_off, rq_cnt; // this step's requests; rq_cnt < 0: evaluate exhaustively
  int state;          // slot state (SLOT_*)
  int m, j1;          // staged motile / hard-sphere joint counts
  int wr;             // bit a: the tile's halo can wrap on axis a
  int unit, gunit;
  const RepParams *rp;
  unsigned long long fb_x, fb_key;  // exhaustive-evaluation result
  double fb_dv;
  double fb_k[3];
};

struct Res {
  unsigned long long xb, key;
  double dv;
  double k[3];  // the partner's FP64 position
};

constexpr int RQ_PER_TILE = 6;   // request list capacity per tile of the block
// phase A gathers a tile's screening list into its share of the result area
constexpr int FLAT_CAP = RQ_PER_TILE * (int)sizeof(Res) / 2;
// a lane holds at most four requests per step (pq0..pq3); more send the
// tile to the exhaustive evaluation

template <int G>
__device__ __forceinline__ void group_argmin_m(double &bx, uint64_t &bkey, unsigned mask) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    const double ox = __shfl_xor_sync(mask, bx, off);
    const uint64_t ok = __shfl_xor_sync(mask, bkey, off);
    if (better(ox, ok, bx, bkey)) {
      bx = ox;
      bkey = ok;
    }
  }
}

__host__ __device__ __forceinline__ size_t lock_tail_bytes(int NT) {
  return (size_t)NT * sizeof(TileRec) + (size_t)NT * RQ_PER_TILE * (sizeof(int2) + sizeof(Res)) + 16 +
         ECMC_NEV * sizeof(unsigned long long);
}

#define SYS(f) (BATCH ? rp->f : P.f)
#define TSYS(R, f) (BATCH ? (R)->f : P.f)

template <int G, bool BATCH>
__global__ void __launch_bounds__(128, 3) ec_lock_kernel(const ECParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int gl = lane & (G - 1);
  const int gbase = lane & ~(G - 1);
  const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1) << gbase);
  const int NT = blockDim.x / G;
  const int gib = tid / G;
  const int64_t sweep = P.sweep_dev ? *P.sweep_dev : P.sweep;
  const int S = P.stage_cap;
  const int NC = BATCH ? P.ncl_max : P.lg[0] * P.lg[1] * P.lg[2];
  const int MNB = P.m_cap;
  const size_t gbytes = group_bytes(S, 0, MNB, NC);
  Stage st = carve(smem + (size_t)gib * gbytes, S, 0, MNB, NC);
#ifdef ECMC_CHECKED
  st.status = P.status;
  st.nglob = P.n;
#endif
  TileRec *tr = (TileRec *)(smem + (size_t)NT * gbytes);
  int2 *rq = (int2 *)(tr + NT);
  Res *rs = (Res *)(rq + NT * RQ_PER_TILE);
  int *rq_n = (int *)(rs + NT * RQ_PER_TILE);
  int *n_run = rq_n + 1;  // slots with a running EC
  unsigned long long *ev_cnt = (unsigned long long *)(rq_n + 4);  // events by outcome, this block
  const int RQ_CAP = NT * P.rq_per_tile;  // at most NT * RQ_PER_TILE
  const int fl_cap = P.rq_per_tile * (FLAT_CAP / RQ_PER_TILE);

  // ------------------------------------------------------------ tile slots
  // The block keeps NT tile slots busy: a slot whose tile has run its ECs is
  // refilled with the next unit of the launch (a device counter), staged by
  // the slot's own group while the other slots go on.  Slot states:
  enum : int { SLOT_EMPTY = 0, SLOT_FRESH = 1, SLOT_RUN = 2, SLOT_DONE = 3 };
  // the group's current tile
  const RepParams *rp = BATCH ? P.reps : nullptr;
  int unit = 0;
  bool live = false;
  int m = 0, j1 = 0, ns = 0;
  double *Rr = P.r;
  LGrid LG;
  float Wf0 = 0.f, Wf1 = 0.f, Wf2 = 0.f;
  if (gl == 0) {
    tr[gib].state = SLOT_EMPTY;
    tr[gib].active = 0;
    tr[gib].rq_cnt = 0;
  }
  if (tid == 0) {
    *rq_n = 0;
    *n_run = 0;
  }
  if (tid < ECMC_NEV) ev_cnt[tid] = 0;
  __syncthreads();

  // take the next unit and stage it (group-collective); false when none left
  auto take_tile = [&]() -> bool {
    int u = 0;
    if (gl == 0) {
      u = atomicAdd(P.unit_next, 1);
      if (P.defer_mode == 2) u = u < *P.n_deferred ? P.deferred[u] : P.n_units;
    }
    u = __shfl_sync(gmask, u, gbase);
    if (u >= P.n_units) return false;
    const int gu = u;
    unit = gu;
    if (BATCH) {
      int lo = 0, hi = P.n_reps - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.reps[mid].unit_off <= gu) lo = mid;
        else hi = mid - 1;
      }
      rp = P.reps + lo;
      unit = gu - (int)rp->unit_off;
    }
    Rr = BATCH ? P.r + 3 * rp->bead_off : P.r;
#ifdef ECMC_CHECKED
    if (BATCH) st.nglob = rp->n_beads;
#endif
    const int32_t *const Rstart = BATCH ? P.cstart + rp->cell_off : P.cstart;
    const uint64_t Rkey = BATCH ? rp->replica : P.replica;
    LG.g0 = SYS(lg)[0];
    LG.g1 = SYS(lg)[1];
    LG.g2 = SYS(lg)[2];
    LG.org = SYS(lorg);
    LG.inv0 = SYS(linv)[0];
    LG.inv1 = SYS(linv)[1];
    LG.inv2 = SYS(linv)[2];
    Wf0 = (float)SYS(W)[0];
    Wf1 = (float)SYS(W)[1];
    Wf2 = (float)SYS(W)[2];
    const int tk0 = unit % SYS(D)[0];
    const int tk1 = (unit / SYS(D)[0]) % SYS(D)[1];
    const int tk2 = unit / (SYS(D)[0] * SYS(D)[1]);
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)sweep, 0, 0, P.seed, Rkey);
    const double c0 = unit53(w.v[0]) * SYS(T)[0] + (double)tk0 * SYS(T)[0];
    const double c1 = unit53(w.v[1]) * SYS(T)[1] + (double)tk1 * SYS(T)[1];
    const double c2 = unit53(w.v[2]) * SYS(T)[2] + (double)tk2 * SYS(T)[2];
    live = true;
    bool over = false;
    stage_tile<G, true, BATCH>(P, rp, st, gl, live, unit, c0, c1, c2, Rr, Rstart, S, 0, MNB, NC, LG,
                               m, j1, ns, gmask, P.defer_mode == 1 ? &over : nullptr);
    if (over && gl == 0) {
      const int at = atomicAdd(P.n_deferred, 1);
      P.deferred[CI(at, P.n_units, 32, P.status)] = gu;
    }
    if (!live) m = 0;
    if (gl == 0) {
      TileRec &T = tr[gib];
      T.c[0] = c0;
      T.c[1] = c1;
      T.c[2] = c2;
      T.m = m;
      T.j1 = j1;
      int wr = 0;
      if (!(c0 - P.halo_te > 0.0 && c0 + SYS(W)[0] + P.halo_te < SYS(L)[0])) wr |= 1;
      if (!(c1 - P.halo_te > 0.0 && c1 + SYS(W)[1] + P.halo_te < SYS(L)[1])) wr |= 2;
      if (!(c2 - P.halo_te > 0.0 && c2 + SYS(W)[2] + P.halo_te < SYS(L)[2])) wr |= 4;
      T.wr = wr;
      T.unit = unit;
      T.gunit = gu;
      T.rp = rp;
    }
    return true;
  };

  // ------------------------------------------------------------ owner state
  // thread t < NT owns slot t: its tile's EC state lives in registers
  const bool owner = tid < NT;
  const int ot = owner ? tid : 0;
  const RepParams *orp = nullptr;
  int o_unit = 0, o_gunit = 0, om = 0;
  Stage ost = carve(smem + (size_t)ot * gbytes, S, 0, MNB, NC);
#ifdef ECMC_CHECKED
  ost.status = P.status;
  ost.nglob = P.n;
#endif
  double *oRr = P.r;
  int32_t *oRi = P.img;
  uint64_t oKey = P.replica;
  double oL0 = 0.0, oL1 = 0.0, oL2 = 0.0;
  uint64_t ohb0 = 0, ohb1 = 0, ohb2 = 0;
  bool owr0 = false, owr1 = false, owr2 = false;
  float ocf0 = 0.f, ocf1 = 0.f, ocf2 = 0.f, oLh0 = 0.f, oLh1 = 0.f, oLh2 = 0.f;
  LGrid OLG;
  uint64_t r2 = 0;
  // beads of the owned tile's system (bounds of the checked build)
  auto ost_n = [&]() -> int64_t { return BATCH ? (orp ? orp->n_beads : 0) : P.n; };
  (void)ost_n;
  // the owned slot's new tile
  auto load_tile = [&]() {
    const TileRec &T = tr[ot];
    orp = T.rp;
    o_unit = T.unit;
    o_gunit = T.gunit;
    om = T.m;
    oRr = BATCH ? P.r + 3 * orp->bead_off : P.r;
    oRi = BATCH ? P.img + 3 * orp->bead_off : P.img;
    oKey = BATCH ? orp->replica : P.replica;
#ifdef ECMC_CHECKED
    if (BATCH) ost.nglob = orp->n_beads;
#endif
    oL0 = TSYS(orp, L)[0];
    oL1 = TSYS(orp, L)[1];
    oL2 = TSYS(orp, L)[2];
    ohb0 = dbits(TSYS(orp, half)[0]);
    ohb1 = dbits(TSYS(orp, half)[1]);
    ohb2 = dbits(TSYS(orp, half)[2]);
    owr0 = T.wr & 1;
    owr1 = T.wr & 2;
    owr2 = T.wr & 4;
    ocf0 = (float)T.c[0];
    ocf1 = (float)T.c[1];
    ocf2 = (float)T.c[2];
    oLh0 = 0.5f * (float)oL0;
    oLh1 = 0.5f * (float)oL1;
    oLh2 = 0.5f * (float)oL2;
    OLG.g0 = TSYS(orp, lg)[0];
    OLG.g1 = TSYS(orp, lg)[1];
    OLG.g2 = TSYS(orp, lg)[2];
    OLG.org = TSYS(orp, lorg);
    OLG.inv0 = TSYS(orp, linv)[0];
    OLG.inv1 = TSYS(orp, linv)[1];
    OLG.inv2 = TSYS(orp, linv)[2];
    r2 = (uint64_t)o_unit;
  };
  const int n_ec = P.ecs_per_tile;
  const uint64_t r1 = (uint64_t)sweep;

  int e = 0;
  bool active = false;
  bool o_any = false;  // the slot ran at least one EC
  int p = 0, pid = 0;
  int o_cell = 0;  // local cell of the pivot's shadow
  double q0 = 0.0, q1 = 0.0, q2 = 0.0, v0 = 0.0, v1 = 0.0, v2 = 0.0, xrem = 0.0, lift = 0.0;
  float pf0 = 0.f, pf1 = 0.f, pf2 = 0.f, vf0 = 0.f, vf1 = 0.f, vf2 = 0.f;
  int64_t nev = 0, ncontact = 0;
  u64x4 swr;
  swr.v[0] = swr.v[1] = swr.v[2] = swr.v[3] = 0;
  uint64_t h = 0;
  double lift_all = 0.0, refl_all = 0.0, disp_all = 0.0;
  unsigned long long tried = 0, confirmed = 0, nev_all = 0, ecs_done = 0;
  unsigned exh = 0;  // exhaustive evaluations led by this lane
  unsigned pub = 0;
  // events by outcome: eight 8-bit fields, added to the block's counters
  // every 255 events and at the end
  uint64_t ev_pk = 0;
  unsigned ev_pn = 0;
  auto flush_outcomes = [&]() {
#pragma unroll
    for (int k = 0; k < ECMC_NEV; ++k) {
      const unsigned c = (unsigned)(ev_pk >> (8 * k)) & 0xFFu;
      if (c) atomicAdd(&ev_cnt[k], (unsigned long long)c);
    }
    ev_pk = 0;
    ev_pn = 0;
  };

  // start EC e of the owned tile: start bead and direction (Sec. II, R6)
  auto start_ec = [&]() {
    const uint64_t r0 = TAG_START | ((uint64_t)e << 8);
    u64x4 w = philox(r0, r1, r2, 0, P.seed, oKey);
    p = (int)scale_below(w.v[0], (uint64_t)om);
    if (P.dir_mode == ECMC_DIR_CART3) {
      const int ax = (int)scale_below(w.v[1], 3);
      v0 = ax == 0 ? 1.0 : 0.0;
      v1 = ax == 1 ? 1.0 : 0.0;
      v2 = ax == 2 ? 1.0 : 0.0;
    } else {
      double a = 2.0 * unit53(w.v[1]) - 1.0;
      double b = 2.0 * unit53(w.v[2]) - 1.0;
      double c = 2.0 * unit53(w.v[3]) - 1.0;
      uint64_t att = 0;
      for (;;) {
        const double s = a * a + b * b + c * c;
        if (s > 1e-6 && s <= 1.0) {
          const double nr = sqrt(s);
          v0 = a / nr;
          v1 = b / nr;
          v2 = c / nr;
          break;
        }
        ++att;
        w = philox(r0, r1, r2, att, P.seed, oKey);
        a = 2.0 * unit53(w.v[0]) - 1.0;
        b = 2.0 * unit53(w.v[1]) - 1.0;
        c = 2.0 * unit53(w.v[2]) - 1.0;
      }
    }
    p = CI(p, om, 10, P.status);
    pid = CI(ost.id[p], ost_n(), 11, P.status);
    q0 = oRr[3 * (int64_t)pid];
    q1 = oRr[3 * (int64_t)pid + 1];
    q2 = oRr[3 * (int64_t)pid + 2];
    pf0 = ost.fx[p];
    pf1 = ost.fy[p];
    pf2 = ost.fz[p];
    {
      int c0, c1, c2;
      o_cell = lcell(OLG, pf0, pf1, pf2, c0, c1, c2);
    }
    vf0 = (float)v0;
    vf1 = (float)v1;
    vf2 = (float)v2;
    xrem = P.ell;
    lift = 0.0;
    nev = 0;
    ncontact = 0;
    swr.v[0] = swr.v[1] = swr.v[2] = swr.v[3] = 0;
    h = 0xCBF29CE484222325ull;
    active = true;
    pub = 3;
  };
  // publish the owned tile's state for the next step
  // (pub: what else changed since the last publish, 1 the direction, 2 the
  // pivot slot)
  auto publish = [&]() {
    TileRec &T = tr[ot];
    T.active = active ? 1 : 0;
    if (!active) return;
    T.q[0] = q0;
    T.q[1] = q1;
    T.q[2] = q2;
    T.pf[0] = pf0;
    T.pf[1] = pf1;
    T.pf[2] = pf2;
    T.xcap = dbits(P.s_cap) < dbits(xrem) ? P.s_cap_f : __double2float_ru(xrem);
    if (pub & 1) {
      T.v[0] = v0;
      T.v[1] = v1;
      T.v[2] = v2;
      T.vf[0] = vf0;
      T.vf[1] = vf1;
      T.vf[2] = vf2;
      T.vnz = (nonzero(v0) ? 1 : 0) | (nonzero(v1) ? 2 : 0) | (nonzero(v2) ? 4 : 0);
    }
    if (pub & 2) T.p = p;
    pub = 0;
  };
  // The pivot's shadow and local cell in the staging area serve only the
  // other beads' screens (a pivot never screens itself), so they are
  // brought up to date when the bead stops being the pivot.
  auto settle_pivot = [&](float f0, float f1, float f2) {
    int c0, c1, c2;
    const int nc = lcell(OLG, f0, f1, f2, c0, c1, c2);
    if (nc != o_cell) {
      lcell_remove(ost, o_cell, p);
      if (!lcell_insert(ost, nc, p)) set_status(P.status, DEV_CAPACITY);
      o_cell = nc;
    }
    ost.fx[p] = f0;
    ost.fy[p] = f1;
    ost.fz[p] = f2;
  };
  // FP32 screen constants
  Screen Z;
  Z.sig2f = (float)P.sig2;
  Z.eps_v = P.eps_v;
  Z.eps_d = P.eps_d;
  {
    const float reach = (float)(P.s_cap + P.sigma + 0.01 * P.sigma);
    Z.near2 = reach * reach;
  }
  const float b2f = (float)P.b2;
  const float eps_v = P.eps_v, eps_d = P.eps_d;
  const float reach_hs = (float)P.sigma + 2.f * eps_v;  // per-axis reach of a contact
  const float INF = __int_as_float(0x7f800000);
  constexpr int ITEMS = G >= 8 ? 1 : 2;  // special candidates per lane
  // the cells of the 27-cell stencil this lane gathers, 7 bits each:
  // offsets dx | dy << 2 | dz << 4 from the stencil's corner, bit 6 set
  constexpr int CPL = (27 + G - 1) / G;  // cells per lane
  using CpkT = typename std::conditional<(7 * CPL <= 32), unsigned, uint64_t>::type;
  CpkT cpk = 0;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int ci = gl + j * G;
    if (ci < 27) cpk |= (CpkT)((ci % 3) | ((ci / 3 % 3) << 2) | ((ci / 9) << 4) | 64) << (7 * j);
  }

  // One step per iteration.  Owners publish their tile's state at the end
  // of the step; the barrier that closes it also tells whether a slot has
  // run out of ECs, and only then do the slots refill.
  bool refill = true;  // every slot starts empty
  for (;;) {
    if (refill) {
      // refill empty slots (each by its own group; tiles without motile
      // beads have no ECs and are passed over)
      if (tr[gib].state == SLOT_EMPTY) {
        for (;;) {
          if (!take_tile()) {
            live = false;
            if (gl == 0) tr[gib].state = SLOT_DONE;
            break;
          }
          if (live && m > 0) {
            if (gl == 0) tr[gib].state = SLOT_FRESH;
            break;
          }
        }
      }
      __syncthreads();
      if (owner && tr[ot].state == SLOT_FRESH) {
        load_tile();
        e = 0;
        o_any = true;
        start_ec();
        tr[ot].state = SLOT_RUN;
        publish();
        atomicAdd(n_run, 1);
      }
      __syncthreads();
    }
    if (*n_run == 0) break;

    // ---------------------------------------------------------- A: screen
    {
      const TileRec &T = tr[gib];
      const bool act = live && T.active;
      int a_p = 0;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
      unsigned nbw = 0xFFFFFFFFu;
      int vnz = 0;
      float ubl = INF;
      if (act) {
        a_p = T.p;
        a0 = T.pf[0];
        a1 = T.pf[1];
        a2 = T.pf[2];
        w0 = T.vf[0];
        w1 = T.vf[1];
        w2 = T.vf[2];
        vnz = T.vnz;
        nbw = st.nb[a_p];
        if (gl == 0) ubl = T.xcap;
      }
      int spk[ITEMS], sps[ITEMS];
      float spl[ITEMS];
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        spk[r] = -1;
        sps[r] = -1;
        spl[r] = INF;
        const int it = gl + r * G;
        if (!act || it == 0 || it >= 6) continue;
        if (it <= 2) {
          int t = it == 1 ? nb_prev(nbw) : nb_next(nbw);
          if (t < 0) continue;
          t = CI(t, S, 20, P.status);
          const float d0 = a0 - st.fx[t], d1 = a1 - st.fy[t], d2 = a2 - st.fz[t];
          const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
          const float dv = __fmaf_rn(d2, w2, __fmaf_rn(d1, w1, d0 * w0));
          const float rad = b2f - (dd - dv * dv);
          const float lo = -dv - eps_v + sqrt_lo(fmaxf(rad - eps_d, 0.f));
          const float hi = -dv + eps_v + sqrt_hi(fmaxf(rad + eps_d, 0.f));
          spl[r] = fmaxf(lo, 0.f);
          ubl = fminf(ubl, fmaxf(hi, 0.f) + 1e-6f);
          spk[r] = KIND_TETHER;
          sps[r] = t;
        } else {
          const int a = it - 3;
          if (!((vnz >> a) & 1)) continue;
          const float vfa = a == 0 ? w0 : (a == 1 ? w1 : w2);
          const float pfa = a == 0 ? a0 : (a == 1 ? a1 : a2);
          const float Wfa = a == 0 ? Wf0 : (a == 1 ? Wf1 : Wf2);
          const float dist = signbit(vfa) ? pfa : Wfa - pfa;
          const float av = fabsf(vfa);
          if (av >= 1e-30f) {
            spl[r] = div_lo(fmaxf(dist - eps_v, 0.f), av);
            ubl = fminf(ubl, div_hi(fmaxf(dist, 0.f) + eps_v, av));
          } else {
            spl[r] = 0.f;  // |v_a| below FP32 range: evaluate in FP64
          }
          spk[r] = KIND_WALL;
          sps[r] = a;
        }
      }
      // gather the slots of the 27 local cells around the pivot and of the
      // overflow list into one list (in the group's share of the result
      // area, which phase B fills only after this phase), then screen it G
      // lanes wide, two slots per lane and round
      unsigned short *fl = reinterpret_cast<unsigned short *>(rs) + gib * FLAT_CAP;
      int pc0 = 0, pc1 = 0, pc2 = 0;
      lcell(LG, a0, a1, a2, pc0, pc1, pc2);
      // only the cells the pivot can reach this step: a hard-sphere partner
      // lies within sigma (plus the screen's margin) of the path
      // [pf, pf + xcap vf] on every axis, a box of one to three cells per
      // axis inside the 27 around the pivot (cells are at least
      // s_cap + 1.012 sigma wide)
      int lo0, lo1, lo2, hi0, hi1, hi2;
      {
        const float xc = act ? T.xcap : 0.f;
        const float e0 = xc * w0, e1 = xc * w1, e2 = xc * w2;
        lcell(LG, a0 - reach_hs + fminf(e0, 0.f), a1 - reach_hs + fminf(e1, 0.f),
              a2 - reach_hs + fminf(e2, 0.f), lo0, lo1, lo2);
        lcell(LG, a0 + reach_hs + fmaxf(e0, 0.f), a1 + reach_hs + fmaxf(e1, 0.f),
              a2 + reach_hs + fmaxf(e2, 0.f), hi0, hi1, hi2);
        lo0 = max(lo0, pc0 - 1);
        lo1 = max(lo1, pc1 - 1);
        lo2 = max(lo2, pc2 - 1);
        hi0 = min(hi0, pc0 + 1);
        hi1 = min(hi1, pc1 + 1);
        hi2 = min(hi2, pc2 + 1);
      }
      const int n_ovf = act ? st.hdr[4] : 0;
      // the box relative to the stencil's corner cell (pc - 1 on every axis)
      const int r0 = lo0 - pc0 + 1, r1 = lo1 - pc1 + 1, r2 = lo2 - pc2 + 1;
      const unsigned n0 = hi0 - lo0, n1 = hi1 - lo1, n2 = hi2 - lo2;
      const int g01 = LG.g0 * LG.g1;
      const int cb = (pc2 - 1) * g01 + (pc1 - 1) * LG.g0 + (pc0 - 1);
      int cw[CPL];  // cell index << 3 | bead count
      int cnt_l = 0;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const unsigned d = (unsigned)(cpk >> (7 * j)) & 127u;
        cw[j] = 0;
        if (!act || !(d & 64u)) continue;
        const int dx = d & 3u, dy = (d >> 2) & 3u, dz = (d >> 4) & 3u;
        if ((unsigned)(dx - r0) > n0 || (unsigned)(dy - r1) > n1 || (unsigned)(dz - r2) > n2) continue;
        const int c = CI(cb + dz * g01 + dy * LG.g0 + dx, NC, 22, P.status);
        const int n = cell_n(st.cell + 8 * c);
        cw[j] = (c << 3) | n;
        cnt_l += n;
      }
      int cincl = cnt_l;
#pragma unroll
      for (int off = 1; off < G; off <<= 1) {
        const int y = __shfl_up_sync(FULL, cincl, off, G);
        if (gl >= off) cincl += y;
      }
      const int ncell = __shfl_sync(FULL, cincl, G - 1, G);
      const int nfl = ncell + n_ovf;
      const bool fl_full = nfl > fl_cap;  // the tile is evaluated exhaustively
      if (!fl_full) {
        int at = cincl - cnt_l;
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
          const int n = cw[j] & 7;
          if (n == 0) continue;
          const uint4 c = *reinterpret_cast<const uint4 *>(st.cell + 8 * (cw[j] >> 3));
          const unsigned short sl[6] = {(unsigned short)(c.y & 0xFFFF), (unsigned short)(c.y >> 16),
                                        (unsigned short)(c.z & 0xFFFF), (unsigned short)(c.z >> 16),
                                        (unsigned short)(c.w & 0xFFFF), (unsigned short)(c.w >> 16)};
#pragma unroll
          for (int i = 0; i < 6; ++i)
            if (i < n) fl[CI(at + i, fl_cap, 23, P.status)] = sl[i];
          at += n;
        }
        for (int i = gl; i < n_ovf; i += G) fl[ncell + i] = st.ovf[i];
      }
      __syncwarp();
      const int nscr = fl_full ? 0 : nfl;
      int ks0 = -1, ks1 = -1;
      float kl0 = INF, kl1 = INF;
      bool kovf = false;
      for (int j = gl; j < nscr; j += 2 * G) {
        const int ka = CI(fl[j], S, 21, P.status);
        const bool two = j + G < nscr;
        const int kb = two ? CI(fl[j + G], S, 21, P.status) : ka;
        const float ax = st.fx[ka], ay = st.fy[ka], az = st.fz[ka];
        const float bx = st.fx[kb], by = st.fy[kb], bz = st.fz[kb];
        if (ka != a_p) screen_hs(Z, a0 - ax, a1 - ay, a2 - az, w0, w1, w2, ka, ubl, ks0, kl0, ks1, kl1, kovf);
        if (two && kb != a_p)
          screen_hs(Z, a0 - bx, a1 - by, a2 - bz, w0, w1, w2, kb, ubl, ks0, kl0, ks1, kl1, kovf);
      }
      const float U = group_minf<G>(ubl);
      // survivors of this lane (kind << 28 | slot)
      int pq0 = 0, pq1 = 0, pq2 = 0, pq3 = 0;
      int npush = 0;
      bool over = act && fl_full;
      auto push = [&](int code) {
        if (npush == 0) pq0 = code;
        else if (npush == 1) pq1 = code;
        else if (npush == 2) pq2 = code;
        else if (npush == 3) pq3 = code;
        else over = true;
        ++npush;
      };
#pragma unroll
      for (int r = 0; r < ITEMS; ++r)
        if (spk[r] >= 0 && spl[r] <= U) push((spk[r] << 28) | sps[r]);
      if (ks0 >= 0 && kl0 <= U) push((KIND_HS << 28) | ks0);
      if (ks1 >= 0 && kl1 <= U) push((KIND_HS << 28) | ks1);
      if (act && kovf) {
        // more than two possible winners in this lane: screen its slots again
        // against the group's U and keep every one that can reach it
        for (int j = gl; j < nscr; j += G) {
          const int k = CI(fl[j], S, 21, P.status);
          if (k == a_p || k == ks0 || k == ks1) continue;
          bool possible;
          const float lb = screen_lb(Z, a0 - st.fx[k], a1 - st.fy[k], a2 - st.fz[k], w0, w1, w2,
                                     possible);
          if (possible && lb <= U) push((KIND_HS << 28) | k);
        }
      }
      // reserve the group's slots in the request list
      const bool gover = (__ballot_sync(FULL, over) & gmask) != 0;
      int cntl = over ? 0 : npush;
      int incl = cntl;
#pragma unroll
      for (int off = 1; off < G; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off, G);
        if (gl >= off) incl += y;
      }
      const int total = __shfl_sync(FULL, incl, G - 1, G);
      int base = 0;
      if (gl == 0 && act) base = (gover || total == 0) ? 0 : atomicAdd(rq_n, total);
      base = __shfl_sync(FULL, base, 0, G);
      const bool fits = act && !gover && base + total <= RQ_CAP;
      if (act && total > 0 && !gover) {
        if (fits) {
          const int at = CI(base + incl - cntl, RQ_CAP - (cntl > 0 ? cntl - 1 : 0), 24, P.status);
          if (cntl > 0) rq[at] = make_int2(gib, pq0);
          if (cntl > 1) rq[at + 1] = make_int2(gib, pq1);
          if (cntl > 2) rq[at + 2] = make_int2(gib, pq2);
          if (cntl > 3) rq[at + 3] = make_int2(gib, pq3);
        } else {
          // reserved slots inside the list carry no request
          for (int i = base + gl; i < base + total && i < RQ_CAP; i += G) rq[i] = make_int2(-1, 0);
        }
      }
      if (gl == 0 && act) {
        tr[gib].rq_off = fits ? base : 0;
        tr[gib].rq_cnt = fits ? total : (total == 0 && !gover ? 0 : -1);
      }
    }
    __syncthreads();

    // ---------------------------------------------------------- B: FP64
    {
      const int nreq = *rq_n < RQ_CAP ? *rq_n : RQ_CAP;
      for (int i = tid; i < nreq; i += blockDim.x) {
        const int2 r = rq[i];
        Res out;
        out.xb = ~0ull;
        out.key = ~0ull;
        out.dv = 0.0;
        out.k[0] = out.k[1] = out.k[2] = 0.0;
        if (r.x >= 0 && CHK(r.x, NT, 25, P.status)) {
          const TileRec &T = tr[r.x];
          const RepParams *R = T.rp;
          const int kind = r.y >> 28;
          const int k = CI(r.y & 0xFFFFF, S, 26, P.status);
          const double Q0 = T.q[0], Q1 = T.q[1], Q2 = T.q[2];
          const double V0 = T.v[0], V1 = T.v[1], V2 = T.v[2];
          const double L0 = TSYS(R, L)[0], L1 = TSYS(R, L)[1], L2 = TSYS(R, L)[2];
          const bool W0 = T.wr & 1, W1 = T.wr & 2, W2 = T.wr & 4;
          ++confirmed;
          if (kind == KIND_WALL) {
            const int a = k;
            const double va = a == 0 ? V0 : (a == 1 ? V1 : V2);
            const double qa = a == 0 ? Q0 : (a == 1 ? Q1 : Q2);
            const double ca = T.c[a];
            const double La = a == 0 ? L0 : (a == 1 ? L1 : L2);
            const double loc = wrapc(qa - ca, La, dbits(TSYS(R, half)[a]), (T.wr >> a) & 1);
            double x = posv(va) ? (TSYS(R, W)[a] - loc) / va : (0.0 - loc) / va;
            if (neg(x)) x = 0.0;
            out.xb = dbits(x);
            out.key = make_key(KIND_WALL, a, 0);
          } else {
            const bool te = kind == KIND_TETHER;
            Stage sk = carve(smem + (size_t)r.x * gbytes, S, 0, MNB, NC);
#ifdef ECMC_CHECKED
            sk.status = P.status;
            sk.nglob = BATCH ? R->n_beads : P.n;
#endif
            double kx, ky, kz, dv;
            double *const Rk = BATCH ? P.r + 3 * R->bead_off : P.r;
            pos64(sk, Rk, k, false, kx, ky, kz);
            const double x =
                quad_x(te, wrapc(Q0 - kx, L0, dbits(TSYS(R, half)[0]), W0),
                       wrapc(Q1 - ky, L1, dbits(TSYS(R, half)[1]), W1),
                       wrapc(Q2 - kz, L2, dbits(TSYS(R, half)[2]), W2), V0, V1, V2,
                       te ? P.b2 : P.sig2, dv);
            if (!neg(x)) {
              out.xb = dbits(x);
              out.key = make_key(te ? KIND_TETHER : KIND_HS, sk.id[k], k);
              out.dv = dv;
              out.k[0] = kx;
              out.k[1] = ky;
              out.k[2] = kz;
            }
          }
        }
        rs[i] = out;
      }
      // tiles whose survivors did not fit: exhaustive FP64 evaluation by the
      // tile's own group (tethers, walls, every contact in the 27 cells)
      const TileRec &T = tr[gib];
      if (live && T.active && T.rq_cnt < 0) {
        if (gl == 0) ++exh;
        const double Q0 = T.q[0], Q1 = T.q[1], Q2 = T.q[2];
        const double V0 = T.v[0], V1 = T.v[1], V2 = T.v[2];
        const double L0 = SYS(L)[0], L1 = SYS(L)[1], L2 = SYS(L)[2];
        const uint64_t hb0 = dbits(SYS(half)[0]), hb1 = dbits(SYS(half)[1]), hb2 = dbits(SYS(half)[2]);
        const bool W0 = T.wr & 1, W1 = T.wr & 2, W2 = T.wr & 4;
        const int fp = CI(T.p, S, 27, P.status);
        const unsigned nbw = st.nb[fp];
        double bx = __longlong_as_double(0x7ff0000000000000ll);
        uint64_t bkey = ~0ull;
        double bdv = 0.0, bk0 = 0.0, bk1 = 0.0, bk2 = 0.0;
        for (int it = gl; it < 6; it += G) {
          if (it == 0) continue;
          if (it <= 2) {
            const int t = it == 1 ? nb_prev(nbw) : nb_next(nbw);
            if (t < 0) continue;
            double kx, ky, kz, dv;
            pos64(st, Rr, t, false, kx, ky, kz);
            const double x = quad_x(true, wrapc(Q0 - kx, L0, hb0, W0), wrapc(Q1 - ky, L1, hb1, W1),
                                    wrapc(Q2 - kz, L2, hb2, W2), V0, V1, V2, P.b2, dv);
            const uint64_t key = make_key(KIND_TETHER, st.id[t], t);
            if (better(x, key, bx, bkey)) {
              bx = x;
              bkey = key;
              bdv = dv;
              bk0 = kx;
              bk1 = ky;
              bk2 = kz;
            }
          } else {
            const int a = it - 3;
            const double va = a == 0 ? V0 : (a == 1 ? V1 : V2);
            if (!nonzero(va)) continue;
            const double qa = a == 0 ? Q0 : (a == 1 ? Q1 : Q2);
            const double loc = wrapc(qa - T.c[a], SYS(L)[a], dbits(SYS(half)[a]), (T.wr >> a) & 1);
            double x = posv(va) ? (SYS(W)[a] - loc) / va : (0.0 - loc) / va;
            if (neg(x)) x = 0.0;
            const uint64_t key = make_key(KIND_WALL, a, 0);
            if (better(x, key, bx, bkey)) {
              bx = x;
              bkey = key;
            }
          }
        }
        int pc0 = 0, pc1 = 0, pc2 = 0;
        lcell(LG, T.pf[0], T.pf[1], T.pf[2], pc0, pc1, pc2);
        for (int ci = gl; ci < 28; ci += G) {
          int n;
          const unsigned short *lst;
          if (ci == 27) {
            n = st.hdr[4];
            lst = st.ovf;
          } else {
            const int x = pc0 + ci % 3 - 1, y = pc1 + (ci / 3) % 3 - 1, z = pc2 + ci / 9 - 1;
            if (x < 0 || y < 0 || z < 0 || x >= LG.g0 || y >= LG.g1 || z >= LG.g2) continue;
            const unsigned short *c = st.cell + 8 * ((z * LG.g1 + y) * LG.g0 + x);
            n = cell_n(c);
            lst = c + 2;
          }
          for (int i = 0; i < n; ++i) {
            const int k = CI(lst[i], S, 28, P.status);
            if (k == fp) continue;
            double kx, ky, kz, dv;
            pos64(st, Rr, k, false, kx, ky, kz);
            const double x = quad_x(false, wrapc(Q0 - kx, L0, hb0, W0), wrapc(Q1 - ky, L1, hb1, W1),
                                    wrapc(Q2 - kz, L2, hb2, W2), V0, V1, V2, P.sig2, dv);
            ++confirmed;
            if (!neg(x)) {
              const uint64_t key = make_key(KIND_HS, st.id[k], k);
              if (better(x, key, bx, bkey)) {
                bx = x;
                bkey = key;
                bdv = dv;
                bk0 = kx;
                bk1 = ky;
                bk2 = kz;
              }
            }
          }
        }
        const uint64_t my_key = bkey;
        const uint64_t my_x = dbits(bx);
        group_argmin_m<G>(bx, bkey, gmask);
        const unsigned own = __ballot_sync(gmask, my_key == bkey && my_x == dbits(bx)) & gmask;
        const int src = __ffs(own) - 1;
        const int from = src < 0 ? lane : src;
        const double wdv = __shfl_sync(gmask, bdv, from);
        const double wk0 = __shfl_sync(gmask, bk0, from);
        const double wk1 = __shfl_sync(gmask, bk1, from);
        const double wk2 = __shfl_sync(gmask, bk2, from);
        if (gl == 0) {
          tr[gib].fb_x = dbits(bx);
          tr[gib].fb_key = bkey;
          tr[gib].fb_dv = wdv;
          tr[gib].fb_k[0] = wk0;
          tr[gib].fb_k[1] = wk1;
          tr[gib].fb_k[2] = wk2;
        }
      }
    }
    __syncthreads();

    // ---------------------------------------------------------- D: move
    if (owner && active && nev >= P.event_cap) {
      set_status(P.status, DEV_STUCK);
      active = false;
      oRr[3 * (int64_t)pid] = q0;
      oRr[3 * (int64_t)pid + 1] = q1;
      oRr[3 * (int64_t)pid + 2] = q2;
      settle_pivot(pf0, pf1, pf2);
    }
    if (owner && active) {
      double x;
      uint64_t bkey;
      double wdv = 0.0, wk0 = 0.0, wk1 = 0.0, wk2 = 0.0;
      {
        const TileRec &T = tr[ot];
        if (dbits(P.s_cap) < dbits(xrem)) {
          x = P.s_cap;
          bkey = make_key(KIND_PASS, 0, 0);
        } else {
          x = xrem;
          bkey = make_key(KIND_END, 0, 0);
        }
        if (T.rq_cnt < 0) {
          const double fx = __longlong_as_double((long long)T.fb_x);
          if (better(fx, T.fb_key, x, bkey)) {
            x = fx;
            bkey = T.fb_key;
            wdv = T.fb_dv;
            wk0 = T.fb_k[0];
            wk1 = T.fb_k[1];
            wk2 = T.fb_k[2];
          }
        } else {
          const int i0 = T.rq_off, i1 = T.rq_off + T.rq_cnt;
          int wi = -1;
          for (int i = i0; i < i1; ++i) {
            if (!CHK(i, RQ_CAP, 29, P.status)) break;
            const unsigned long long xb = rs[i].xb, kb = rs[i].key;
            if (xb < dbits(x) || (xb == dbits(x) && kb < bkey)) {
              x = __longlong_as_double((long long)xb);
              bkey = kb;
              wi = i;
            }
          }
          if (wi >= 0) {
            wdv = rs[wi].dv;
            wk0 = rs[wi].k[0];
            wk1 = rs[wi].k[1];
            wk2 = rs[wi].k[2];
          }
        }
      }
      const int kind = key_kind(bkey);
      const int slot = CI(key_slot(bkey), S, 30, P.status);
      const int64_t partner = (kind == KIND_END || kind == KIND_PASS) ? -1 : key_id(bkey);
      int di0 = 0, di1 = 0, di2 = 0;
      if (owr0) di0 = step_i(q0, x, v0, oL0);
      else q0 = __fma_rn(x, v0, q0);
      if (owr1) di1 = step_i(q1, x, v1, oL1);
      else q1 = __fma_rn(x, v1, q1);
      if (owr2) di2 = step_i(q2, x, v2, oL2);
      else q2 = __fma_rn(x, v2, q2);
      if (di0 | di1 | di2) {
        if (di0) oRi[3 * (int64_t)pid] += di0;
        if (di1) oRi[3 * (int64_t)pid + 1] += di1;
        if (di2) oRi[3 * (int64_t)pid + 2] += di2;
      }
      ++nev;
      int out;
      bool swapped = false;
      double sw0 = 0.0, sw1 = 0.0, sw2 = 0.0;  // the partner's position after a swap
      int np = p;
      if (kind == KIND_END) {
        out = ECMC_EV_END;
      } else if (kind == KIND_PASS) {
        out = ECMC_EV_PASS;
      } else if (kind == KIND_WALL) {
        out = ECMC_EV_WALL;
        pub |= 1;
        // (negation is exact in both precisions)
        if (partner == 0) {
          v0 = -v0;
          vf0 = -vf0;
        } else if (partner == 1) {
          v1 = -v1;
          vf1 = -vf1;
        } else {
          v2 = -v2;
          vf2 = -vf2;
        }
      } else {
        // (r_target - r_pivot).v at contact = -(d.v) - x
        const double proj = -wdv - x;
        const bool motile = slot < om;
        if (!motile) {
          out = kind == KIND_HS ? ECMC_EV_HS_REFLECT : ECMC_EV_TE_REFLECT;
          refl_all = refl_all + proj;
          pub |= 1;
          mirror2(v0, v1, v2, wrapc(q0 - wk0, oL0, ohb0, owr0), wrapc(q1 - wk1, oL1, ohb1, owr1),
                  wrapc(q2 - wk2, oL2, ohb2, owr2));
          vf0 = (float)v0;
          vf1 = (float)v1;
          vf2 = (float)v2;
        } else if (kind == KIND_HS) {
          lift = lift + proj;
          if (P.swap_mode) {
            bool go;
            if (P.swap_mode == 1) {
              go = true;
            } else {
              if ((ncontact & 3) == 0)
                swr = philox(TAG_SWAP | ((uint64_t)e << 8), r1, r2, (uint64_t)(ncontact >> 2), P.seed,
                             oKey);
              go = (swr.v[ncontact & 3] >> 11) < P.swap_thr;
            }
            ++ncontact;
            if (go) {
              ++tried;
              const double k0 = wk0, k1 = wk1, k2 = wk2;
              // every bond of both beads, positions exchanged, within b_max
              bool ok = true;
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const int a = side == 0 ? p : slot;
                const double a0 = side == 0 ? k0 : q0;
                const double a1 = side == 0 ? k1 : q1;
                const double a2 = side == 0 ? k2 : q2;
                const unsigned nbv = ost.nb[a];
#pragma unroll
                for (int dir = 0; dir < 2; ++dir) {
                  const int b = dir == 0 ? nb_prev(nbv) : nb_next(nbv);
                  if (b < 0) continue;
                  double b0, b1, b2;
                  if (b == p) {
                    b0 = k0;
                    b1 = k1;
                    b2 = k2;
                  } else if (b == slot) {
                    b0 = q0;
                    b1 = q1;
                    b2 = q2;
                  } else {
                    pos64(ost, oRr, b, false, b0, b1, b2);
                  }
                  const double e0 = wrapc(a0 - b0, oL0, ohb0, owr0);
                  const double e1 = wrapc(a1 - b1, oL1, ohb1, owr1);
                  const double e2 = wrapc(a2 - b2, oL2, ohb2, owr2);
                  const double dd = __fma_rn(e2, e2, __fma_rn(e1, e1, e0 * e0));
                  ok = ok && !(dbits(dd) > dbits(P.b2));
                }
              }
              if (ok) {
                swapped = true;
                const int kid = ost.id[slot];
                oRr[3 * (int64_t)kid] = q0;
                oRr[3 * (int64_t)kid + 1] = q1;
                oRr[3 * (int64_t)kid + 2] = q2;
                sw0 = q0;
                sw1 = q1;
                sw2 = q2;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  const int ti = oRi[3 * (int64_t)pid + a];
                  oRi[3 * (int64_t)pid + a] = oRi[3 * (int64_t)kid + a];
                  oRi[3 * (int64_t)kid + a] = ti;
                }
                q0 = k0;
                q1 = k1;
                q2 = k2;
              }
            }
          }
          if (swapped) {
            out = ECMC_EV_SWAP;
          } else {
            out = ECMC_EV_HS_LIFT;
            np = slot;
          }
        } else {
          lift = lift + proj;
          out = ECMC_EV_TE_LIFT;
          np = slot;
        }
      }
      ev_pk += 1ull << (8 * out);
      if (++ev_pn == 255) flush_outcomes();
      // FP32 shadow of the moved pivot: FP32 position minus FP32 corner
      float nf0 = (float)q0 - ocf0, nf1 = (float)q1 - ocf1, nf2 = (float)q2 - ocf2;
      if (owr0) nf0 = nf0 > oLh0 ? nf0 - (float)oL0 : (nf0 < -oLh0 ? nf0 + (float)oL0 : nf0);
      if (owr1) nf1 = nf1 > oLh1 ? nf1 - (float)oL1 : (nf1 < -oLh1 ? nf1 + (float)oL1 : nf1);
      if (owr2) nf2 = nf2 > oLh2 ? nf2 - (float)oL2 : (nf2 < -oLh2 ? nf2 + (float)oL2 : nf2);
      if (P.rec_digest) {
        fnv_mix(h, (uint64_t)pid);
        fnv_mix(h, ((uint64_t)(uint32_t)out << 32) | (uint64_t)(uint32_t)partner);
        fnv_mix(h, dbits(x));
      }
      if (P.log) {
        const unsigned long long at = atomicAdd(P.log_n, 1ull);
        if ((int64_t)at < P.log_cap) {
          ecmc_event ev;
          ev.unit = P.rec_offset + (P.sweep_dev ? (sweep - P.rec_sweep0) * P.n_units * n_ec : 0) +
                    (int64_t)o_gunit * n_ec + e;
          ev.seq = (int32_t)(nev - 1);
          ev.pivot = pid;
          ev.kind = out;
          ev.pad = 0;
          ev.partner = partner;
          ev.x = x;
          P.log[at] = ev;
        }
      }
      if (out == ECMC_EV_END || np != p) {
        // the pivot's FP64 position stays in registers while it is the
        // pivot (no other thread reads it) and goes back to the global
        // array when the EC ends or is handed on
        oRr[3 * (int64_t)pid] = q0;
        oRr[3 * (int64_t)pid + 1] = q1;
        oRr[3 * (int64_t)pid + 2] = q2;
      }
      if (swapped) {
        // the partner takes the pivot's old position: its shadow and local cell
        float g0 = (float)sw0 - ocf0, g1 = (float)sw1 - ocf1, g2 = (float)sw2 - ocf2;
        if (owr0) g0 = g0 > oLh0 ? g0 - (float)oL0 : (g0 < -oLh0 ? g0 + (float)oL0 : g0);
        if (owr1) g1 = g1 > oLh1 ? g1 - (float)oL1 : (g1 < -oLh1 ? g1 + (float)oL1 : g1);
        if (owr2) g2 = g2 > oLh2 ? g2 - (float)oL2 : (g2 < -oLh2 ? g2 + (float)oL2 : g2);
        int a0, a1, a2;
        const int koc = lcell(OLG, ost.fx[slot], ost.fy[slot], ost.fz[slot], a0, a1, a2);
        const int knc = lcell(OLG, g0, g1, g2, a0, a1, a2);
        if (koc != knc) {
          lcell_remove(ost, koc, slot);
          if (!lcell_insert(ost, knc, slot)) set_status(P.status, DEV_CAPACITY);
        }
        ost.fx[slot] = g0;
        ost.fy[slot] = g1;
        ost.fz[slot] = g2;
      }
      if (out == ECMC_EV_END || np != p) settle_pivot(nf0, nf1, nf2);
      pf0 = nf0;
      pf1 = nf1;
      pf2 = nf2;
      if (out == ECMC_EV_END) {
        active = false;
      } else {
        xrem = xrem - x;
      }
      if (active && np != p) {
        // lift: the partner (motile, unmoved this event) becomes the pivot
        p = np;
        pub |= 2;
        pid = CI(ost.id[p], ost_n(), 31, P.status);
        q0 = wk0;
        q1 = wk1;
        q2 = wk2;
        pf0 = ost.fx[p];
        pf1 = ost.fy[p];
        pf2 = ost.fz[p];
        int c0, c1, c2;
        o_cell = lcell(OLG, pf0, pf1, pf2, c0, c1, c2);
      }
    }
    // end of an EC: records, then the tile's next EC or a new tile
    if (owner && tr[ot].state == SLOT_RUN && !active) {
      lift_all = lift_all + lift;
      disp_all = disp_all + P.ell;  // the free flights of an EC add up to ell
      nev_all += (unsigned long long)nev;
      ++ecs_done;
      if (P.rec_digest) {
        const int64_t idx = P.rec_offset + (P.sweep_dev ? (sweep - P.rec_sweep0) * P.n_units * n_ec : 0) +
                            (int64_t)o_gunit * n_ec + e;
        if (idx < P.rec_cap) {
          P.rec_digest[idx] = h;
          P.rec_lift[idx] = lift;
          P.rec_events[idx] = nev;
        }
      }
      ++e;
      if (e < n_ec) {
        start_ec();
      } else {
        tr[ot].state = SLOT_EMPTY;
        atomicSub(n_run, 1);
      }
    }
    if (owner) publish();
    if (tid == 0) *rq_n = 0;
    refill = __syncthreads_or(owner && tr[ot].state == SLOT_EMPTY);
  }

  // ------------------------------------------------------------ counters
  if (confirmed) atomicAdd(&P.counters[CNT_CONFIRMED], confirmed);
  if (exh) atomicAdd(&P.counters[CNT_EXHAUSTIVE], (unsigned long long)exh);
  if (ev_pn) flush_outcomes();
  __syncthreads();
  if (tid < ECMC_NEV && ev_cnt[tid]) atomicAdd(&P.counters[tid], ev_cnt[tid]);
  if (o_any && ecs_done) {
    atomicAdd(&P.counters[CNT_EVENTS], nev_all);
    if (tried) atomicAdd(&P.counters[CNT_SWAP_TRIED], tried);
    atomicAdd(&P.counters[CNT_ECS], ecs_done);
    atomicAdd(&P.sums[SUM_LIFT], lift_all);
    atomicAdd(&P.sums[SUM_REFL], refl_all);
    atomicAdd(&P.sums[SUM_DISP], disp_all);
  }
}
#undef TSYS
#undef SYS

}  // namespace

size_t lock_smem_bytes(int stage_cap, int motile_cap, int ncell, int tiles_per_block) {
  return (size_t)tiles_per_block * group_bytes(stage_cap, 0, motile_cap, ncell) +
         lock_tail_bytes(tiles_per_block);
}

// tiles per block and resident blocks for one capacity setting (memoised)
struct LockShape {
  size_t key = 0;
  int nt = 0, blocks = 0;
};

template <int G, bool BATCH>
static cudaError_t lock_shape(const ECParams &P, int S, int M, int NC, LockShape *memo, int *nt_out,
                              int *res_out, size_t *smem_out) {
  static int smem_max = 0;
  if (!smem_max) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(ec_lock_kernel<G, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_max);
    if (e != cudaSuccess) return e;
  }
  const size_t key = (lock_smem_bytes(S, M, NC, 1) * 64 + (size_t)P.block_tiles) * 4096 +
                     (size_t)(P.n_units % 4096);
  for (int i = 0; i < 2; ++i) {
    if (memo[i].key == key && memo[i].nt) {
      *nt_out = memo[i].nt;
      *res_out = memo[i].blocks;
      *smem_out = lock_smem_bytes(S, M, NC, memo[i].nt);
      return cudaSuccess;
    }
  }
  // tiles per block: whole warps, at most 32 (the owners fill warp 0) and
  // 128 threads; among those, the most tiles resident per SM
  const int step = 32 / G > 1 ? 32 / G : 1;
  int nt = 0, best = -1, best_blocks = 0;
  for (int t = step; t <= 32 && t * G <= 128; t += step) {
    if (P.block_tiles > 0 && t != P.block_tiles) continue;
    const size_t sm = lock_smem_bytes(S, M, NC, t);
    if (sm > (size_t)smem_max) break;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ec_lock_kernel<G, BATCH>, t * G, sm) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    if (blocks * t > best) {
      best = blocks * t;
      nt = t;
      best_blocks = blocks;
    }
  }
  if (nt == 0 || best_blocks < 1) return cudaErrorInvalidValue;
  memo[1] = memo[0];
  memo[0].key = key;
  memo[0].nt = nt;
  memo[0].blocks = best_blocks;
  *nt_out = nt;
  *res_out = best_blocks;
  *smem_out = lock_smem_bytes(S, M, NC, nt);
  return cudaSuccess;
}

template <int G, bool BATCH>
static cudaError_t launch_lock_t(const ECParams &P0, cudaStream_t s) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  static LockShape memo[2];
  const int NC = BATCH ? P0.ncl_max : P0.lg[0] * P0.lg[1] * P0.lg[2];
  const bool two = P0.stage_tight > 0 && P0.m_tight > 0 && P0.deferred && P0.n_deferred &&
                   (P0.stage_tight < P0.stage_cap || P0.m_tight < P0.m_cap);
  // persistent blocks: as many as stay resident, each pulling tiles from the
  // unit counter until none are left
  auto run = [&](ECParams P, int S, int M, int mode) -> cudaError_t {
    P.stage_cap = S;
    P.m_cap = M;
    P.defer_mode = mode;
    int nt = 0, res = 0;
    size_t smem = 0;
    cudaError_t e = lock_shape<G, BATCH>(P, S, M, NC, memo, &nt, &res, &smem);
    if (e != cudaSuccess) return e;
    const long long want = (P.n_units + nt - 1) / nt;
    const long long room = (long long)res * sms;
    const int blocks = (int)(want < room ? want : room);
    e = cudaMemsetAsync(P.unit_next, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (blocks > 0) ec_lock_kernel<G, BATCH><<<blocks, nt * G, smem, s>>>(P);
    return cudaGetLastError();
  };
  if (!two) return run(P0, P0.stage_cap, P0.m_cap, 0);
  cudaError_t e = cudaMemsetAsync(P0.n_deferred, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  e = run(P0, P0.stage_tight, P0.m_tight, 1);
  if (e != cudaSuccess) return e;
  return run(P0, P0.stage_cap, P0.m_cap, 2);
}

cudaError_t launch_ec_lock(const ECParams &P, int lanes, cudaStream_t s) {
  if (!P.domain) return cudaErrorInvalidValue;
  if (P.k_spring != 0.0) return cudaErrorInvalidValue;  // bead springs: k_ec.cu
  if (lanes == 8) return launch_lock_t<8, false>(P, s);
  if (lanes == 4) return launch_lock_t<4, false>(P, s);
  if (lanes == 16) return launch_lock_t<16, false>(P, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_ec_lock_batch(const ECParams &P, int lanes, cudaStream_t s) {
  if (lanes == 8) return launch_lock_t<8, true>(P, s);
  if (lanes == 4) return launch_lock_t<4, true>(P, s);
  if (lanes == 16) return launch_lock_t<16, true>(P, s);
  return cudaErrorInvalidValue;
}

}  // namespace ecmc
