// Event-chain kernel, one lane per tile (arXiv:1502.06447, Sec. II: EC
// move; Sec. II.B: tile-joint decomposition with reflections; Sec. II.D:
// swap move).
//
// Each thread runs the ECs of one tile on its own; the 32 tiles of a warp
// advance through the same code in SIMT lockstep, so every instruction — the
// FP64 ones included — serves 32 tiles, and no lane waits on another.
//
// Per sweep the thread stages its tile into a private scratch region in
// global memory (L2-resident for the workloads here): every bead within the
// tether halo of the tile, with an FP32 tile-local shadow and its id, the
// motile beads' slots sorted by id (start beads: slot mot[below(u, m)]), the
// bond partners of motile beads, and a local cell grid of side >= the reach
// of one free flight (s_cap + sigma) and >= b_max, kept current as beads
// move.  An event reads the 27 cells around the pivot.  FP64 positions stay
// in the global position array (joint beads are static during a sweep;
// motile beads are written only by their tile's thread).
//
// The screened form (F32) bounds every candidate in FP32 and evaluates in
// FP64 only those whose lower bound can reach the smallest upper bound U; the
// plain form evaluates every candidate of the 27 cells in FP64.  Both give
// the event sequence of the plain definition (a candidate outside the 27
// cells is farther than one free flight).
#include <cuda_runtime.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ bool neg(double x) {
  const uint64_t b = dbits(x);
  return (int64_t)b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool posv(double x) { return (int64_t)dbits(x) > 0; }
__device__ __forceinline__ bool ge_pos(double y, double L) {
  return (int64_t)dbits(y) >= (int64_t)dbits(L);
}
__device__ __forceinline__ bool nonzero(double x) { return (dbits(x) << 1) != 0; }
__device__ __forceinline__ double wrap_i(double d, double L, uint64_t hbits) {
  const uint64_t b = dbits(d);
  if ((b & 0x7FFFFFFFFFFFFFFFull) > hbits) return ((int64_t)b < 0) ? d + L : d - L;
  return d;
}
__device__ __forceinline__ int step_i(double &r, double x, double v, double L) {
  double y = __fma_rn(x, v, r);
  int di = 0;
  if (ge_pos(y, L)) {
    y = y - L;
    di = 1;
  } else if (neg(y)) {
    y = y + L;
    di = -1;
    if (ge_pos(y, L)) {
      y = 0.0;
      di = 0;
    }
  }
  r = y;
  return di;
}
// contact (tether = false, R2 = sigma^2) or tether limit (R2 = b_max^2)
__device__ __forceinline__ double quad_x(bool tether, double d0, double d1, double d2, double v0,
                                         double v1, double v2, double R2, double &dv) {
  dv = __fma_rn(d2, v2, __fma_rn(d1, v1, d0 * v0));
  if (!tether && !neg(dv)) return -1.0;
  const double dd = __fma_rn(d2, d2, __fma_rn(d1, d1, d0 * d0));
  double rad = R2 - __fma_rn(-dv, dv, dd);
  if (tether) {
    if (neg(rad)) rad = 0.0;
  } else if (!posv(rad)) {
    return -1.0;
  }
  const double x = tether ? -dv + sqrt(rad) : -dv - sqrt(rad);
  return neg(x) ? 0.0 : x;
}
__device__ __forceinline__ void mirror2(double &v0, double &v1, double &v2, double d0, double d1,
                                        double d2) {
  const double dd = __fma_rn(d2, d2, __fma_rn(d1, d1, d0 * d0));
  const double vd = __fma_rn(v2, d2, __fma_rn(v1, d1, v0 * d0));
  const double t = (2.0 * vd) / dd;
  v0 = __fma_rn(-t, d0, v0);
  v1 = __fma_rn(-t, d1, v1);
  v2 = __fma_rn(-t, d2, v2);
}
// tie order within equal x: (kind, partner id)
__device__ __forceinline__ bool better(double x, int kind, int64_t id, double bx, int bkind,
                                       int64_t bid) {
  const uint64_t a = dbits(x), b = dbits(bx);
  return a < b || (a == b && (kind < bkind || (kind == bkind && id < bid)));
}
__device__ __forceinline__ void set_status(int *st, int code) { atomicCAS(st, 0, code); }

// ---------------------------------------------------------------- scratch
constexpr int CELL_CAP = 7;     // slots per local cell (16 B: count + 7)
constexpr int ID_MASK = (1 << 29) - 1;
constexpr int ID_MOTILE = 1 << 30;
constexpr int OVF_CAP = 64;     // beads of over-full cells, always scanned

struct Tile {
  float4 *sh;        // [S] shadow xyz (tile-local), w = id | motile << 30 (bits)
  unsigned *nb;      // [S] bond partner slots, 16 + 16 bits, 0xFFFF = none
  unsigned short *mot;  // [S] motile slots sorted by id
  uint4 *cell;       // [NC] count (low 16 of .x) + 7 slots
  unsigned short *ovf;  // [OVF_CAP]
  int *ovf_n;
};

__device__ __forceinline__ Tile tile_at(unsigned char *base, int S, int NC) {
  Tile t;
  t.sh = (float4 *)base;
  t.nb = (unsigned *)(t.sh + S);
  t.mot = (unsigned short *)(t.nb + S);
  size_t off = (size_t)S * 16 + (size_t)S * 4 + (((size_t)S * 2 + 15) / 16) * 16;
  t.cell = (uint4 *)(base + off);
  t.ovf = (unsigned short *)(t.cell + NC);
  t.ovf_n = (int *)(t.ovf + OVF_CAP);
  return t;
}

__device__ __forceinline__ int cell_count(const uint4 &c) { return (int)(c.x & 0xFFFF); }
__device__ __forceinline__ int cell_slot(const uint4 &c, int i) {
  const unsigned w = i == 0 ? (c.x >> 16)
                   : i == 1 ? (c.y & 0xFFFF)
                   : i == 2 ? (c.y >> 16)
                   : i == 3 ? (c.z & 0xFFFF)
                   : i == 4 ? (c.z >> 16)
                   : i == 5 ? (c.w & 0xFFFF)
                            : (c.w >> 16);
  return (int)(w & 0xFFFF);
}
__device__ __forceinline__ void cell_set(uint4 &c, int i, int s) {
  const unsigned v = (unsigned)s & 0xFFFF;
  if (i == 0) c.x = (c.x & 0xFFFF) | (v << 16);
  else if (i == 1) c.y = (c.y & 0xFFFF0000u) | v;
  else if (i == 2) c.y = (c.y & 0xFFFF) | (v << 16);
  else if (i == 3) c.z = (c.z & 0xFFFF0000u) | v;
  else if (i == 4) c.z = (c.z & 0xFFFF) | (v << 16);
  else if (i == 5) c.w = (c.w & 0xFFFF0000u) | v;
  else c.w = (c.w & 0xFFFF) | (v << 16);
}

struct Grid {
  int g0, g1, g2;
  float org;             // local coordinate of the grid's low corner (all axes)
  float inv0, inv1, inv2;  // cells per unit length
};

__device__ __forceinline__ int cell_index(const Grid &G, float f0, float f1, float f2, int &c0,
                                          int &c1, int &c2) {
  c0 = (int)((f0 - G.org) * G.inv0);
  c1 = (int)((f1 - G.org) * G.inv1);
  c2 = (int)((f2 - G.org) * G.inv2);
  c0 = c0 < 0 ? 0 : (c0 >= G.g0 ? G.g0 - 1 : c0);
  c1 = c1 < 0 ? 0 : (c1 >= G.g1 ? G.g1 - 1 : c1);
  c2 = c2 < 0 ? 0 : (c2 >= G.g2 ? G.g2 - 1 : c2);
  return (c2 * G.g1 + c1) * G.g0 + c0;
}

__device__ __forceinline__ bool cell_insert(const Tile &T, int ci, int slot) {
  uint4 c = T.cell[ci];
  const int n = cell_count(c);
  if (n < CELL_CAP) {
    cell_set(c, n, slot);
    c.x = (c.x & 0xFFFF0000u) | (unsigned)(n + 1);
    T.cell[ci] = c;
    return true;
  }
  const int k = *T.ovf_n;
  if (k >= OVF_CAP) return false;
  T.ovf[k] = (unsigned short)slot;
  *T.ovf_n = k + 1;
  return true;
}

__device__ __forceinline__ void cell_remove(const Tile &T, int ci, int slot) {
  uint4 c = T.cell[ci];
  const int n = cell_count(c);
  for (int i = 0; i < n; ++i) {
    if (cell_slot(c, i) == slot) {
      cell_set(c, i, cell_slot(c, n - 1));
      c.x = (c.x & 0xFFFF0000u) | (unsigned)(n - 1);
      T.cell[ci] = c;
      return;
    }
  }
  const int k = *T.ovf_n;
  for (int i = 0; i < k; ++i) {
    if (T.ovf[i] == slot) {
      T.ovf[i] = T.ovf[k - 1];
      *T.ovf_n = k - 1;
      return;
    }
  }
}

template <bool F32>
__global__ void __launch_bounds__(64) ec_lane_kernel(const ECParams P) {
  const int unit = blockIdx.x * blockDim.x + threadIdx.x;
  if (unit >= P.n_units) return;
  const int S = P.stage_cap;
  const int NC = P.lg[0] * P.lg[1] * P.lg[2];
  Tile T = tile_at(P.scratch + (size_t)unit * (size_t)P.tile_bytes, S, NC);
  Grid G;
  G.g0 = P.lg[0];
  G.g1 = P.lg[1];
  G.g2 = P.lg[2];
  G.org = P.lorg;
  G.inv0 = P.linv[0];
  G.inv1 = P.linv[1];
  G.inv2 = P.linv[2];
  const uint64_t hb0 = dbits(P.half[0]), hb1 = dbits(P.half[1]), hb2 = dbits(P.half[2]);
  const int tx = unit % P.D[0], ty = (unit / P.D[0]) % P.D[1], tz = unit / (P.D[0] * P.D[1]);
  double c0, c1, c2;
  {
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)P.sweep, 0, 0, P.seed, P.replica);
    c0 = unit53(w.v[0]) * P.T[0] + (double)tx * P.T[0];
    c1 = unit53(w.v[1]) * P.T[1] + (double)ty * P.T[1];
    c2 = unit53(w.v[2]) * P.T[2] + (double)tz * P.T[2];
  }

  // ------------------------------------------------------------ staging
  for (int i = 0; i < NC; ++i) T.cell[i] = make_uint4(0, 0, 0, 0);
  *T.ovf_n = 0;
  int ns = 0, m = 0;
  bool bad = false;
  {
    const double corner[3] = {c0, c1, c2};
    int c_lo[3], c_n[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lo = corner[a] - P.halo_te, hi = corner[a] + P.W[a] + P.halo_te;
      int l = (int)floor(lo / P.cs[a]);
      const int h = (int)floor(hi / P.cs[a]);
      int cnt = h - l + 1;
      if (cnt >= P.nc[a]) {
        l = 0;
        cnt = P.nc[a];
      }
      c_lo[a] = l;
      c_n[a] = cnt;
    }
    for (int qz = 0; qz < c_n[2]; ++qz) {
      int cz = (c_lo[2] + qz) % P.nc[2];
      if (cz < 0) cz += P.nc[2];
      for (int qy = 0; qy < c_n[1]; ++qy) {
        int cy = (c_lo[1] + qy) % P.nc[1];
        if (cy < 0) cy += P.nc[1];
        for (int qx = 0; qx < c_n[0]; ++qx) {
          int cx = (c_lo[0] + qx) % P.nc[0];
          if (cx < 0) cx += P.nc[0];
          const int cell = (cz * P.nc[1] + cy) * P.nc[0] + cx;
          const int j0 = P.cstart[cell], jend = P.cstart[cell + 1];
          for (int j = j0; j < jend; ++j) {
            const int tg = P.ctag[j];
            if (tg != unit && tg >= 0) continue;  // another tile's bead
            const double s0 = wrap_i(P.cr[3 * (int64_t)j] - c0, P.L[0], hb0);
            const double s1 = wrap_i(P.cr[3 * (int64_t)j + 1] - c1, P.L[1], hb1);
            const double s2 = wrap_i(P.cr[3 * (int64_t)j + 2] - c2, P.L[2], hb2);
            if (tg < 0) {
              const bool in = s0 >= -P.halo_te && s0 <= P.W[0] + P.halo_te && s1 >= -P.halo_te &&
                              s1 <= P.W[1] + P.halo_te && s2 >= -P.halo_te &&
                              s2 <= P.W[2] + P.halo_te;
              if (!in) continue;
            }
            if (ns >= S) {
              bad = true;
              continue;
            }
            const int id = P.cid[j];
            const float f0 = (float)s0, f1 = (float)s1, f2 = (float)s2;
            T.sh[ns] = make_float4(f0, f1, f2, __int_as_float(id | (tg == unit ? ID_MOTILE : 0)));
            T.nb[ns] = 0xFFFFFFFFu;
            int a0, a1, a2;
            if (!cell_insert(T, cell_index(G, f0, f1, f2, a0, a1, a2), ns)) bad = true;
            if (tg == unit) {
              // insertion into the id-sorted motile list
              int k = m;
              while (k > 0) {
                const int prev = T.mot[k - 1];
                if ((__float_as_int(T.sh[prev].w) & ID_MASK) < id) break;
                T.mot[k] = (unsigned short)prev;
                --k;
              }
              T.mot[k] = (unsigned short)ns;
              ++m;
            }
            ++ns;
          }
        }
      }
    }
  }
  if (bad) {
    set_status(P.status, DEV_CAPACITY);
    return;
  }
  // bond partners of motile beads: within b_max, so in the 27 cells around
  for (int k = 0; k < m; ++k) {
    const int s = T.mot[k];
    const float4 me = T.sh[s];
    const int id = __float_as_int(me.w) & ID_MASK;
    const int c = id % P.N;
    const int want_p = c != 0 ? id - 1 : -1;
    const int want_n = c != P.N - 1 ? id + 1 : -1;
    int fp = -1, fn = -1;
    int a0, a1, a2;
    cell_index(G, me.x, me.y, me.z, a0, a1, a2);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = a0 + dx, y = a1 + dy, z = a2 + dz;
          if (x < 0 || y < 0 || z < 0 || x >= G.g0 || y >= G.g1 || z >= G.g2) continue;
          const uint4 cc = T.cell[(z * G.g1 + y) * G.g0 + x];
          const int n = cell_count(cc);
          for (int i = 0; i < n; ++i) {
            const int t = cell_slot(cc, i);
            const int tid = __float_as_int(T.sh[t].w) & ID_MASK;
            if (tid == want_p) fp = t;
            if (tid == want_n) fn = t;
          }
        }
    for (int i = 0; i < *T.ovf_n; ++i) {
      const int t = T.ovf[i];
      const int tid = __float_as_int(T.sh[t].w) & ID_MASK;
      if (tid == want_p) fp = t;
      if (tid == want_n) fn = t;
    }
    if ((want_p >= 0 && fp < 0) || (want_n >= 0 && fn < 0)) set_status(P.status, DEV_TILE);
    T.nb[s] = ((unsigned)(fn < 0 ? 0xFFFF : fn) << 16) | (unsigned)(fp < 0 ? 0xFFFF : fp);
  }
  if (m == 0) return;

  // ------------------------------------------------------------ ECs
  const float sig2f = (float)P.sig2;
  const float b2f = (float)P.b2;
  const float eps_v = P.eps_v, eps_d = P.eps_d;
  const float reach = (float)(P.s_cap + P.sigma + 0.01 * P.sigma);
  const float near2 = reach * reach;
  const float Wf0 = (float)P.W[0], Wf1 = (float)P.W[1], Wf2 = (float)P.W[2];
  const float INF = __int_as_float(0x7f800000);
  const double DINF = __longlong_as_double(0x7ff0000000000000ll);
  double lift_all = 0.0, refl_all = 0.0, disp_all = 0.0;
  unsigned long long cnt[ECMC_NEV];
#pragma unroll
  for (int k = 0; k < ECMC_NEV; ++k) cnt[k] = 0;
  unsigned long long tried = 0, confirmed = 0, nev_all = 0;
  const int n_ec = P.ecs_per_tile;

  for (int e = 0; e < n_ec; ++e) {
    const uint64_t r0 = TAG_START | ((uint64_t)e << 8);
    const uint64_t r1 = (uint64_t)P.sweep;
    const uint64_t r2 = (uint64_t)unit;
    double v0, v1, v2;
    int p;
    {
      u64x4 w = philox(r0, r1, r2, 0, P.seed, P.replica);
      p = T.mot[(int)scale_below(w.v[0], (uint64_t)m)];
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
          w = philox(r0, r1, r2, att, P.seed, P.replica);
          a = 2.0 * unit53(w.v[0]) - 1.0;
          b = 2.0 * unit53(w.v[1]) - 1.0;
          c = 2.0 * unit53(w.v[2]) - 1.0;
        }
      }
    }
    float4 pme = T.sh[p];
    int pid = __float_as_int(pme.w) & ID_MASK;
    double q0 = P.r[3 * (int64_t)pid], q1 = P.r[3 * (int64_t)pid + 1], q2 = P.r[3 * (int64_t)pid + 2];
    float vf0 = (float)v0, vf1 = (float)v1, vf2 = (float)v2;
    double xrem = P.ell;
    int64_t nev = 0, ncontact = 0;
    u64x4 swr;
    swr.v[0] = swr.v[1] = swr.v[2] = swr.v[3] = 0;
    uint64_t h = 0xCBF29CE484222325ull;
    double lift = 0.0;
    bool active = true;
    while (active) {
      if (nev >= P.event_cap) {
        set_status(P.status, DEV_STUCK);
        break;
      }
      const float pf0 = pme.x, pf1 = pme.y, pf2 = pme.z;
      const unsigned nbw = T.nb[p];
      // best exactly evaluated candidate; END / PASS first
      double bx;
      int bkind;
      int64_t bid = -1;
      int bslot = -1;
      double bdv = 0.0;
      if (dbits(P.s_cap) < dbits(xrem)) {
        bx = P.s_cap;
        bkind = KIND_PASS;
      } else {
        bx = xrem;
        bkind = KIND_END;
      }
      float U = F32 ? __double2float_ru(bx) : 0.f;
      // survivors awaiting FP64 confirmation (slot | tether << 16), walls apart
      float wall_lb[3] = {INF, INF, INF};
      int keep_s[4];
      float keep_l[4];
      int nk = 0;
      bool ovf_keep = false;
      if (F32) {
        // tethers
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const unsigned tw = side == 0 ? (nbw & 0xFFFF) : (nbw >> 16);
          if (tw == 0xFFFF) continue;
          const float4 o = T.sh[tw];
          const float d0 = pf0 - o.x, d1 = pf1 - o.y, d2 = pf2 - o.z;
          const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
          const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
          const float rad = b2f - (dd - dv * dv);
          const float lo = -dv - eps_v + sqrt_lo(fmaxf(rad - eps_d, 0.f));
          const float hi = -dv + eps_v + sqrt_hi(fmaxf(rad + eps_d, 0.f));
          U = fminf(U, fmaxf(hi, 0.f) + 1e-6f);
          keep_s[nk] = (int)tw | (1 << 16);
          keep_l[nk] = fmaxf(lo, 0.f);
          ++nk;
        }
        // walls
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const double va = a == 0 ? v0 : (a == 1 ? v1 : v2);
          if (!nonzero(va)) continue;
          const float vfa = a == 0 ? vf0 : (a == 1 ? vf1 : vf2);
          const float pfa = a == 0 ? pf0 : (a == 1 ? pf1 : pf2);
          const float Wfa = a == 0 ? Wf0 : (a == 1 ? Wf1 : Wf2);
          const float dist = posv(va) ? Wfa - pfa : pfa;
          const float av = fabsf(vfa);
          if (av >= 1e-30f) {
            wall_lb[a] = div_lo(fmaxf(dist - eps_v, 0.f), av);
            U = fminf(U, div_hi(fmaxf(dist, 0.f) + eps_v, av));
          } else {
            wall_lb[a] = 0.f;
          }
        }
      }
      // hard-sphere obstacles in the 27 cells around the pivot (+ overflow)
      int a0, a1, a2;
      cell_index(G, pf0, pf1, pf2, a0, a1, a2);
      const int n_ovf = *T.ovf_n;
      for (int ci = -1; ci < 27; ++ci) {
        uint4 cc;
        int n;
        if (ci < 0) {
          n = n_ovf;
        } else {
          const int x = a0 + ci % 3 - 1, y = a1 + (ci / 3) % 3 - 1, z = a2 + ci / 9 - 1;
          if (x < 0 || y < 0 || z < 0 || x >= G.g0 || y >= G.g1 || z >= G.g2) continue;
          cc = T.cell[(z * G.g1 + y) * G.g0 + x];
          n = cell_count(cc);
        }
        for (int i = 0; i < n; ++i) {
          const int k = ci < 0 ? (int)T.ovf[i] : cell_slot(cc, i);
          if (k == p) continue;
          const float4 o = T.sh[k];
          if (!F32) {
            const int kid = __float_as_int(o.w) & ID_MASK;
            double dv;
            const double x = quad_x(false, wrap_i(q0 - P.r[3 * (int64_t)kid], P.L[0], hb0),
                                    wrap_i(q1 - P.r[3 * (int64_t)kid + 1], P.L[1], hb1),
                                    wrap_i(q2 - P.r[3 * (int64_t)kid + 2], P.L[2], hb2), v0, v1,
                                    v2, P.sig2, dv);
            if (!neg(x) && better(x, KIND_HS, kid, bx, bkind, bid)) {
              bx = x;
              bkind = KIND_HS;
              bid = kid;
              bslot = k;
              bdv = dv;
            }
            continue;
          }
          const float d0 = pf0 - o.x, d1 = pf1 - o.y, d2 = pf2 - o.z;
          const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
          if (dd > near2) continue;
          const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
          const float disc = sig2f - (dd - dv * dv);
          if (!(dv < eps_v && disc > -eps_d)) continue;
          if (dv < -eps_v && disc > eps_d)
            U = fminf(U, fmaxf(0.f, -dv + eps_v - sqrt_lo(disc - eps_d)) + 1e-6f);
          const float lb = -dv - eps_v - sqrt_hi(disc + eps_d);
          if (lb > U) continue;
          // keep: drop entries that U has already excluded, then append
          int w = 0;
          for (int t = 0; t < nk; ++t)
            if (keep_l[t] <= U) {
              keep_s[w] = keep_s[t];
              keep_l[w] = keep_l[t];
              ++w;
            }
          nk = w;
          if (nk < 4) {
            keep_s[nk] = k;
            keep_l[nk] = lb;
            ++nk;
          } else {
            ovf_keep = true;
          }
        }
      }
      if (F32) {
        // FP64 confirmation of every candidate whose lower bound reaches U
        for (int t = 0; t < nk; ++t) {
          if (keep_l[t] > U) continue;
          const bool te = (keep_s[t] >> 16) & 1;
          const int k = keep_s[t] & 0xFFFF;
          const int kid = __float_as_int(T.sh[k].w) & ID_MASK;
          double dv;
          const double x = quad_x(te, wrap_i(q0 - P.r[3 * (int64_t)kid], P.L[0], hb0),
                                  wrap_i(q1 - P.r[3 * (int64_t)kid + 1], P.L[1], hb1),
                                  wrap_i(q2 - P.r[3 * (int64_t)kid + 2], P.L[2], hb2), v0, v1, v2,
                                  te ? P.b2 : P.sig2, dv);
          ++confirmed;
          const int kd = te ? KIND_TETHER : KIND_HS;
          if (!neg(x) && better(x, kd, kid, bx, bkind, bid)) {
            bx = x;
            bkind = kd;
            bid = kid;
            bslot = k;
            bdv = dv;
          }
        }
        if (ovf_keep) {
          // more than four possible winners: evaluate the 27 cells again
          for (int ci = -1; ci < 27; ++ci) {
            uint4 cc;
            int n;
            if (ci < 0) {
              n = n_ovf;
            } else {
              const int x = a0 + ci % 3 - 1, y = a1 + (ci / 3) % 3 - 1, z = a2 + ci / 9 - 1;
              if (x < 0 || y < 0 || z < 0 || x >= G.g0 || y >= G.g1 || z >= G.g2) continue;
              cc = T.cell[(z * G.g1 + y) * G.g0 + x];
              n = cell_count(cc);
            }
            for (int i = 0; i < n; ++i) {
              const int k = ci < 0 ? (int)T.ovf[i] : cell_slot(cc, i);
              if (k == p) continue;
              const float4 o = T.sh[k];
              const float d0 = pf0 - o.x, d1 = pf1 - o.y, d2 = pf2 - o.z;
              const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
              if (dd > near2) continue;
              const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
              const float disc = sig2f - (dd - dv * dv);
              const float lb = -dv - eps_v - sqrt_hi(disc + eps_d);
              if (!(dv < eps_v && disc > -eps_d && lb <= U)) continue;
              const int kid = __float_as_int(o.w) & ID_MASK;
              double dvx;
              const double x = quad_x(false, wrap_i(q0 - P.r[3 * (int64_t)kid], P.L[0], hb0),
                                      wrap_i(q1 - P.r[3 * (int64_t)kid + 1], P.L[1], hb1),
                                      wrap_i(q2 - P.r[3 * (int64_t)kid + 2], P.L[2], hb2), v0,
                                      v1, v2, P.sig2, dvx);
              ++confirmed;
              if (!neg(x) && better(x, KIND_HS, kid, bx, bkind, bid)) {
                bx = x;
                bkind = KIND_HS;
                bid = kid;
                bslot = k;
                bdv = dvx;
              }
            }
          }
        }
      } else {
        // plain FP64: tethers exactly
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const unsigned tw = side == 0 ? (nbw & 0xFFFF) : (nbw >> 16);
          if (tw == 0xFFFF) continue;
          const int kid = __float_as_int(T.sh[tw].w) & ID_MASK;
          double dv;
          const double x = quad_x(true, wrap_i(q0 - P.r[3 * (int64_t)kid], P.L[0], hb0),
                                  wrap_i(q1 - P.r[3 * (int64_t)kid + 1], P.L[1], hb1),
                                  wrap_i(q2 - P.r[3 * (int64_t)kid + 2], P.L[2], hb2), v0, v1, v2,
                                  P.b2, dv);
          if (better(x, KIND_TETHER, kid, bx, bkind, bid)) {
            bx = x;
            bkind = KIND_TETHER;
            bid = kid;
            bslot = (int)tw;
            bdv = dv;
          }
        }
      }
      // walls (FP64 when the screen lets them through, always in plain FP64)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double va = a == 0 ? v0 : (a == 1 ? v1 : v2);
        if (!nonzero(va)) continue;
        if (F32 && !(wall_lb[a] <= U)) continue;
        const double qa = a == 0 ? q0 : (a == 1 ? q1 : q2);
        const double ca = a == 0 ? c0 : (a == 1 ? c1 : c2);
        const double loc = wrap_i(qa - ca, P.L[a], a == 0 ? hb0 : (a == 1 ? hb1 : hb2));
        double x = posv(va) ? (P.W[a] - loc) / va : (0.0 - loc) / va;
        if (neg(x)) x = 0.0;
        if (F32) ++confirmed;
        if (better(x, KIND_WALL, a, bx, bkind, bid)) {
          bx = x;
          bkind = KIND_WALL;
          bid = a;
        }
      }

      // ---------------- apply the event
      const double x = bx;
      const int64_t partner = (bkind == KIND_END || bkind == KIND_PASS) ? -1 : bid;
      const int di0 = step_i(q0, x, v0, P.L[0]);
      const int di1 = step_i(q1, x, v1, P.L[1]);
      const int di2 = step_i(q2, x, v2, P.L[2]);
      if (di0 | di1 | di2) {
        if (di0) P.img[3 * (int64_t)pid] += di0;
        if (di1) P.img[3 * (int64_t)pid + 1] += di1;
        if (di2) P.img[3 * (int64_t)pid + 2] += di2;
      }
      ++nev;
      int out;
      int np = p;
      bool swapped = false;
      if (bkind == KIND_END) {
        out = ECMC_EV_END;
      } else if (bkind == KIND_PASS) {
        out = ECMC_EV_PASS;
      } else if (bkind == KIND_WALL) {
        out = ECMC_EV_WALL;
        if (bid == 0) v0 = -v0;
        else if (bid == 1) v1 = -v1;
        else v2 = -v2;
      } else {
        const double proj = -bdv - x;
        const int64_t kid = bid;
        const double k0 = P.r[3 * kid], k1 = P.r[3 * kid + 1], k2 = P.r[3 * kid + 2];
        const bool mot = (__float_as_int(T.sh[bslot].w) & ID_MOTILE) != 0;
        if (!mot) {
          out = bkind == KIND_HS ? ECMC_EV_HS_REFLECT : ECMC_EV_TE_REFLECT;
          refl_all = refl_all + proj;
          mirror2(v0, v1, v2, wrap_i(q0 - k0, P.L[0], hb0), wrap_i(q1 - k1, P.L[1], hb1),
                  wrap_i(q2 - k2, P.L[2], hb2));
        } else if (bkind == KIND_HS) {
          lift = lift + proj;
          if (P.swap_mode) {
            bool go;
            if (P.swap_mode == 1) {
              go = true;
            } else {
              if ((ncontact & 3) == 0)
                swr = philox(TAG_SWAP | ((uint64_t)e << 8), r1, r2, (uint64_t)(ncontact >> 2),
                             P.seed, P.replica);
              go = (swr.v[ncontact & 3] >> 11) < P.swap_thr;
            }
            ++ncontact;
            if (go) {
              ++tried;
              bool ok = true;
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const int a = side == 0 ? p : bslot;
                const double e0 = side == 0 ? k0 : q0;
                const double e1 = side == 0 ? k1 : q1;
                const double e2 = side == 0 ? k2 : q2;
                const unsigned nbv = T.nb[a];
#pragma unroll
                for (int dir = 0; dir < 2; ++dir) {
                  const unsigned b = dir == 0 ? (nbv & 0xFFFF) : (nbv >> 16);
                  if (b == 0xFFFF) continue;
                  double b0, b1, b2;
                  if ((int)b == p) {
                    b0 = k0;
                    b1 = k1;
                    b2 = k2;
                  } else if ((int)b == bslot) {
                    b0 = q0;
                    b1 = q1;
                    b2 = q2;
                  } else {
                    const int bid2 = __float_as_int(T.sh[b].w) & ID_MASK;
                    b0 = P.r[3 * (int64_t)bid2];
                    b1 = P.r[3 * (int64_t)bid2 + 1];
                    b2 = P.r[3 * (int64_t)bid2 + 2];
                  }
                  const double f0 = wrap_i(e0 - b0, P.L[0], hb0);
                  const double f1 = wrap_i(e1 - b1, P.L[1], hb1);
                  const double f2 = wrap_i(e2 - b2, P.L[2], hb2);
                  const double dd = __fma_rn(f2, f2, __fma_rn(f1, f1, f0 * f0));
                  ok = ok && !(dbits(dd) > dbits(P.b2));
                }
              }
              if (ok) {
                swapped = true;
                // exchange positions, shadows (the cells follow) and images
                P.r[3 * kid] = q0;
                P.r[3 * kid + 1] = q1;
                P.r[3 * kid + 2] = q2;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  const int ti = P.img[3 * (int64_t)pid + a];
                  P.img[3 * (int64_t)pid + a] = P.img[3 * kid + a];
                  P.img[3 * kid + a] = ti;
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
            np = bslot;
          }
        } else {
          lift = lift + proj;
          out = ECMC_EV_TE_LIFT;
          np = bslot;
        }
      }
#pragma unroll
      for (int k = 0; k < ECMC_NEV; ++k) cnt[k] += (out == k);
      fnv_mix(h, (uint64_t)pid);
      fnv_mix(h, ((uint64_t)(uint32_t)out << 32) | (uint64_t)(uint32_t)partner);
      fnv_mix(h, dbits(x));
      if (P.log) {
        const unsigned long long at = atomicAdd(P.log_n, 1ull);
        if ((int64_t)at < P.log_cap) {
          ecmc_event ev;
          ev.unit = P.rec_offset + (int64_t)unit * n_ec + e;
          ev.seq = (int32_t)(nev - 1);
          ev.pivot = pid;
          ev.kind = out;
          ev.pad = 0;
          ev.partner = partner;
          ev.x = x;
          P.log[at] = ev;
        }
      }
      // store the pivot; refresh its shadow and its cell
      P.r[3 * (int64_t)pid] = q0;
      P.r[3 * (int64_t)pid + 1] = q1;
      P.r[3 * (int64_t)pid + 2] = q2;
      {
        const float n0 = (float)wrap_i(q0 - c0, P.L[0], hb0);
        const float n1 = (float)wrap_i(q1 - c1, P.L[1], hb1);
        const float n2 = (float)wrap_i(q2 - c2, P.L[2], hb2);
        int o0, o1, o2, m0, m1, m2;
        const int oc = cell_index(G, pme.x, pme.y, pme.z, o0, o1, o2);
        const int nc = cell_index(G, n0, n1, n2, m0, m1, m2);
        if (swapped) {
          // the pivot took the hit bead's place and vice versa: swap shadows
          const float4 ko = T.sh[bslot];
          const float k0f = (float)wrap_i(P.r[3 * bid] - c0, P.L[0], hb0);
          const float k1f = (float)wrap_i(P.r[3 * bid + 1] - c1, P.L[1], hb1);
          const float k2f = (float)wrap_i(P.r[3 * bid + 2] - c2, P.L[2], hb2);
          int b0, b1, b2, e0, e1, e2;
          const int koc = cell_index(G, ko.x, ko.y, ko.z, b0, b1, b2);
          const int knc = cell_index(G, k0f, k1f, k2f, e0, e1, e2);
          cell_remove(T, koc, bslot);
          cell_remove(T, oc, p);
          T.sh[bslot] = make_float4(k0f, k1f, k2f, ko.w);
          if (!cell_insert(T, knc, bslot)) set_status(P.status, DEV_CAPACITY);
          pme = make_float4(n0, n1, n2, pme.w);
          T.sh[p] = pme;
          if (!cell_insert(T, nc, p)) set_status(P.status, DEV_CAPACITY);
        } else {
          if (oc != nc) {
            cell_remove(T, oc, p);
            if (!cell_insert(T, nc, p)) set_status(P.status, DEV_CAPACITY);
          }
          pme = make_float4(n0, n1, n2, pme.w);
          T.sh[p] = pme;
        }
      }
      if (out == ECMC_EV_END) {
        active = false;
      } else {
        xrem = xrem - x;
        if (out == ECMC_EV_HS_REFLECT || out == ECMC_EV_TE_REFLECT || out == ECMC_EV_WALL) {
          vf0 = (float)v0;
          vf1 = (float)v1;
          vf2 = (float)v2;
        }
        if (np != p) {
          p = np;
          pme = T.sh[p];
          pid = __float_as_int(pme.w) & ID_MASK;
          q0 = P.r[3 * (int64_t)pid];
          q1 = P.r[3 * (int64_t)pid + 1];
          q2 = P.r[3 * (int64_t)pid + 2];
        }
      }
    }
    lift_all = lift_all + lift;
    disp_all = disp_all + P.ell;
    nev_all += (unsigned long long)nev;
    if (P.rec_digest) {
      const int64_t idx = P.rec_offset + (int64_t)unit * n_ec + e;
      if (idx < P.rec_cap) {
        P.rec_digest[idx] = h;
        P.rec_lift[idx] = lift;
        P.rec_events[idx] = nev;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < ECMC_NEV; ++k)
    if (cnt[k]) atomicAdd(&P.counters[k], cnt[k]);
  atomicAdd(&P.counters[CNT_EVENTS], nev_all);
  if (tried) atomicAdd(&P.counters[CNT_SWAP_TRIED], tried);
  if (confirmed) atomicAdd(&P.counters[CNT_CONFIRMED], confirmed);
  atomicAdd(&P.counters[CNT_ECS], (unsigned long long)n_ec);
  atomicAdd(&P.sums[SUM_LIFT], lift_all);
  atomicAdd(&P.sums[SUM_REFL], refl_all);
  atomicAdd(&P.sums[SUM_DISP], disp_all);
}

}  // namespace

size_t lane_tile_bytes(int stage_cap, int ncell) {
  const size_t S = (size_t)stage_cap;
  size_t b = S * 16 + S * 4 + ((S * 2 + 15) / 16) * 16 + (size_t)ncell * 16 + OVF_CAP * 2 + 16;
  return (b + 127) / 128 * 128;
}

cudaError_t launch_ec_lane(const ECParams &P, int fp32f, cudaStream_t s) {
  const int threads = 64;
  const int blocks = (P.n_units + threads - 1) / threads;
  if (fp32f) ec_lane_kernel<true><<<blocks, threads, 0, s>>>(P);
  else ec_lane_kernel<false><<<blocks, threads, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace ecmc
