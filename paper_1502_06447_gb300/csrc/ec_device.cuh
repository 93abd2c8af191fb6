// Device helpers shared by the EC kernels (arXiv:1502.06447, Sec. II, II.A,
// II.C): FP64 comparisons on bit patterns, the minimum image, the contact and
// tether distances (Eq. 1), the reflection (Fig. 2c), candidate keys and the
// tie rule, the shared-memory staging of one tile and its local cell grid,
// and the FP32 screen.  Included by the kernel translation units only.
#pragma once
#include <cuda_runtime.h>
#include <float.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- FP64 bits
__device__ __forceinline__ uint64_t dbits(double x) { return (uint64_t)__double_as_longlong(x); }
// x < 0.0 (false for -0.0)
__device__ __forceinline__ bool neg(double x) {
  const uint64_t b = dbits(x);
  return (int64_t)b < 0 && (b << 1) != 0;
}
// x > 0.0
__device__ __forceinline__ bool posv(double x) { return (int64_t)dbits(x) > 0; }
// y >= L for L > 0
__device__ __forceinline__ bool ge_pos(double y, double L) {
  return (int64_t)dbits(y) >= (int64_t)dbits(L);
}
__device__ __forceinline__ bool nonzero(double x) { return (dbits(x) << 1) != 0; }

// minimum image, same result as d > h ? d - L : (d < -h ? d + L : d)
__device__ __forceinline__ double wrap_i(double d, double L, uint64_t hbits) {
  const uint64_t b = dbits(d);
  if ((b & 0x7FFFFFFFFFFFFFFFull) > hbits) return ((int64_t)b < 0) ? d + L : d - L;
  return d;
}

// wrap_i on an axis that can need it; identity on an axis that cannot
__device__ __forceinline__ double wrapc(double d, double L, uint64_t hbits, bool w) {
  return w ? wrap_i(d, L, hbits) : d;
}

// r += x v on one axis, back into [0, L); returns the image change
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

// Hard-sphere contact (Eq. 1, R2 = sigma^2) or tether limit (R2 = b_max^2)
// of a pivot moving along v, d = pivot - partner.  Returns x >= 0, or -1 when
// a contact candidate misses; dv = d.v.
// (skip_overlap: a hard sphere the pivot overlaps is no obstacle, the
// push-off rule of Sec. II.B)
__device__ __forceinline__ double quad_x(bool tether, double d0, double d1, double d2, double v0,
                                         double v1, double v2, double R2, double &dv,
                                         bool skip_overlap = false) {
  dv = __fma_rn(d2, v2, __fma_rn(d1, v1, d0 * v0));
  if (!tether && !neg(dv)) return -1.0;
  const double dd = __fma_rn(d2, d2, __fma_rn(d1, d1, d0 * d0));
  if (!tether && skip_overlap && dd < R2) return -1.0;
  double rad = R2 - __fma_rn(-dv, dv, dd);
  if (tether) {
    if (neg(rad)) rad = 0.0;
  } else if (!posv(rad)) {
    return -1.0;
  }
  const double x = tether ? -dv + sqrt(rad) : -dv - sqrt(rad);
  return neg(x) ? 0.0 : x;
}

// v <- v - (2 v.d / d.d) d: reflection at the plane normal to d (Fig. 2c)
__device__ __forceinline__ void mirror2(double &v0, double &v1, double &v2, double d0, double d1,
                                        double d2) {
  const double dd = __fma_rn(d2, d2, __fma_rn(d1, d1, d0 * d0));
  const double vd = __fma_rn(v2, d2, __fma_rn(v1, d1, v0 * d0));
  const double t = (2.0 * vd) / dd;
  v0 = __fma_rn(-t, d0, v0);
  v1 = __fma_rn(-t, d1, v1);
  v2 = __fma_rn(-t, d2, v2);
}

// candidate key: kind (3 bits) | partner id (41 bits) | slot (20 bits).
// Key order within equal x = (kind, partner id) order, the tie rule.
__device__ __forceinline__ uint64_t make_key(int kind, int64_t id, int slot) {
  return ((uint64_t)kind << 61) | (((uint64_t)id & ((1ull << 41) - 1)) << 20) |
         (uint64_t)(slot & 0xFFFFF);
}
__device__ __forceinline__ int key_kind(uint64_t k) { return (int)(k >> 61); }
__device__ __forceinline__ int64_t key_id(uint64_t k) { return (int64_t)((k >> 20) & ((1ull << 41) - 1)); }
__device__ __forceinline__ int key_slot(uint64_t k) { return (int)(k & 0xFFFFF); }

// x >= 0 always, so its bit pattern orders like the value
__device__ __forceinline__ bool better(double x, uint64_t key, double bx, uint64_t bkey) {
  const uint64_t a = dbits(x), b = dbits(bx);
  return a < b || (a == b && key < bkey);
}

template <int G>
__device__ __forceinline__ void group_argmin(double &bx, uint64_t &bkey) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    const double ox = __shfl_xor_sync(FULL, bx, off);
    const uint64_t ok = __shfl_xor_sync(FULL, bkey, off);
    if (better(ox, ok, bx, bkey)) {
      bx = ox;
      bkey = ok;
    }
  }
}

template <int G>
__device__ __forceinline__ float group_minf(float v) {
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, off));
  return v;
}

// FP32 minimum image (serial mode only; tile-local shadows need none)
__device__ __forceinline__ float wrapf(float d, float L) {
  return d > 0.5f * L ? d - L : (d < -0.5f * L ? d + L : d);
}

// ---------------------------------------------------------------- staging
// Shared memory of one group: FP64 positions of the first M64 slots (the
// warp-lockstep kernel: M64 = the motile capacity in the screened domain
// form, where joint beads' FP64 positions, static during a sweep, are read
// from the global array when an evaluation needs them, M64 = S otherwise;
// the block-lockstep kernel keeps every FP64 position in the global array,
// M64 = 0); bond-partner words of the first MNB slots (the motile beads);
// FP32 shadow (12 B) and id (4 B) of all S slots; the local cell grid (16 B
// per cell: a 32-bit count, then 6 slots of 16 bits); the overflow list of
// beads whose cell was full; a header.
constexpr int CELL_CAP = 6;
constexpr int OVF_CAP = 64;
constexpr int HDR_BYTES = 32;
// the overflow list holds max(64, S / 4) slots, rounded up to a multiple of
// 8 (16 bytes, so that a group's share of shared memory stays a multiple of
// 16 bytes for any S that is a multiple of 8): clustered inputs (phantom
// chains before the push-off) fill many cells past CELL_CAP
__host__ __device__ __forceinline__ int ovf_cap_for(int S) {
  return S / 4 > OVF_CAP ? (S / 4 + 7) / 8 * 8 : OVF_CAP;
}

struct Stage {
  double *px, *py, *pz;  // [M64]
  unsigned *nb;          // [MNB] bond partner slots, 16 + 16 bits (0xFFFF = none)
  float *fx, *fy, *fz;   // [S]
  int *id;               // [S]
  unsigned short *cell;  // [NC][8]: 32-bit count, then up to 6 slots
  unsigned short *ovf;   // [ovf_cap]
  int *hdr;              // [2] staged count, [3] overflow, [4] overflow-list length
  int ovf_cap;           // ovf_cap_for(S)
#ifdef ECMC_CHECKED
  int cap;               // S (slots)
  long long nglob;       // beads of the system (ids), set by the kernel
  int *status;
#endif
};

__host__ __device__ __forceinline__ size_t group_bytes(int S, int M64, int MNB, int NC) {
  return (size_t)M64 * 24 + (size_t)MNB * 4 + (size_t)S * 16 + (size_t)NC * 16 + (size_t)ovf_cap_for(S) * 2 +
         HDR_BYTES;
}  // (16 B per cell: a 32-bit count and 6 slots of 16 bits)

// S, M64 and MNB are multiples of 8 (capacities are rounded to 8 or 32), so
// every array starts 16-byte aligned and group_bytes is a multiple of 16
__device__ __forceinline__ Stage carve(unsigned char *base, int S, int M64, int MNB, int NC) {
  Stage s;
  s.px = (double *)base;
  s.py = s.px + M64;
  s.pz = s.py + M64;
  s.nb = (unsigned *)(s.pz + M64);
  s.fx = (float *)(s.nb + MNB);
  s.fy = s.fx + S;
  s.fz = s.fy + S;
  s.id = (int *)(s.fz + S);
  s.cell = (unsigned short *)(s.id + S);
  s.ovf = s.cell + 8 * NC;
  s.ovf_cap = ovf_cap_for(S);
  s.hdr = (int *)(s.ovf + s.ovf_cap);
#ifdef ECMC_CHECKED
  s.cap = S;
  s.nglob = 0x7fffffffffffffffll;
  s.status = nullptr;
#endif
  return s;
}

__device__ __forceinline__ int nb_prev(unsigned w) { return (w & 0xFFFF) == 0xFFFF ? -1 : (int)(w & 0xFFFF); }
__device__ __forceinline__ int nb_next(unsigned w) { return (w >> 16) == 0xFFFF ? -1 : (int)(w >> 16); }
__device__ __forceinline__ unsigned nb_pack(int prev, int next) {
  return ((unsigned)(next < 0 ? 0xFFFF : next) << 16) | (unsigned)(prev < 0 ? 0xFFFF : prev);
}

// binary search of id in the sorted range [lo, hi); -1 if absent
__device__ __forceinline__ int find_id(const int *ids, int lo, int hi, int id) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int v = ids[mid];
    if (v == id) return mid;
    if (v < id) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// linear search of id in the unsorted range [lo, hi); -1 if absent
__device__ __forceinline__ int find_id_lin(const int *ids, int lo, int hi, int id) {
  for (int i = lo; i < hi; ++i)
    if (ids[i] == id) return i;
  return -1;
}

__device__ __forceinline__ void set_status(int *st, int code) { atomicCAS(st, 0, code); }

// Bounds checks of the checked build (-DECMC_CHECKED): CHK(i, n, site, st)
// is true when 0 <= i < n; otherwise it records DEV_BOUNDS | site << 8 in
// the status word st (first failure wins) and is false, and the caller
// skips the access.  CI(i, ...) is i, or 0 after a failed check; it
// evaluates i once (the index can be an atomic's result).  In the normal
// build CHK is the constant true and CI the index itself.
#ifdef ECMC_CHECKED
__device__ __forceinline__ bool chk_range(long long i, long long n, int site, int *st) {
  if (i >= 0 && i < n) return true;
  atomicCAS(st, 0, DEV_BOUNDS | (site << 8));
  return false;
}
template <class T>
__device__ __forceinline__ T chk_index(T i, long long n, int site, int *st) {
  return chk_range((long long)i, n, site, st) ? i : T(0);
}
#define CHK(i, n, site, st) chk_range((long long)(i), (long long)(n), (site), (st))
#define CI(i, n, site, st) chk_index((i), (long long)(n), (site), (st))
#else
#define CHK(i, n, site, st) true
#define CI(i, n, site, st) (i)
#endif

// ---------------------------------------------------------------- local grid
struct LGrid {
  int g0, g1, g2;
  float org, inv0, inv1, inv2;
};

__device__ __forceinline__ int lcell(const LGrid &L, float f0, float f1, float f2, int &c0,
                                     int &c1, int &c2) {
  c0 = (int)((f0 - L.org) * L.inv0);
  c1 = (int)((f1 - L.org) * L.inv1);
  c2 = (int)((f2 - L.org) * L.inv2);
  c0 = c0 < 0 ? 0 : (c0 >= L.g0 ? L.g0 - 1 : c0);
  c1 = c1 < 0 ? 0 : (c1 >= L.g1 ? L.g1 - 1 : c1);
  c2 = c2 < 0 ? 0 : (c2 >= L.g2 ? L.g2 - 1 : c2);
  return (c2 * L.g1 + c1) * L.g0 + c0;
}

__device__ __forceinline__ unsigned &cell_count(unsigned short *c) { return *reinterpret_cast<unsigned *>(c); }
__device__ __forceinline__ int cell_n(const unsigned short *c) {
  return (int)*reinterpret_cast<const unsigned *>(c);
}

// single-writer updates (one lane of the group)
__device__ __forceinline__ bool lcell_insert(const Stage &st, int ci, int slot) {
  unsigned short *c = st.cell + 8 * ci;
  const int n = cell_n(c);
  if (n < CELL_CAP) {
    c[2 + n] = (unsigned short)slot;
    cell_count(c) = (unsigned)(n + 1);
    return true;
  }
  const int k = st.hdr[4];
  if (k >= st.ovf_cap) return false;
  st.ovf[k] = (unsigned short)slot;
  st.hdr[4] = k + 1;
  return true;
}

__device__ __forceinline__ void lcell_remove(const Stage &st, int ci, int slot) {
  unsigned short *c = st.cell + 8 * ci;
  const int n = cell_n(c);
  for (int i = 2; i < 2 + n; ++i) {
    if (c[i] == slot) {
      c[i] = c[1 + n];
      cell_count(c) = (unsigned)(n - 1);
      return;
    }
  }
  const int k = st.hdr[4];
  for (int i = 0; i < k; ++i) {
    if (st.ovf[i] == slot) {
      st.ovf[i] = st.ovf[k - 1];
      st.hdr[4] = k - 1;
      return;
    }
  }
}

// FP32 screen of one hard-sphere obstacle k for the pivot shadow pf moving
// along vf: updates the upper bound ubl and keeps the slot when its lower
// bound can reach it (two kept per lane, more -> ovf)
struct Screen {
  float sig2f, eps_v, eps_d, near2;
};

__device__ __forceinline__ void screen_hs(const Screen &Z, float d0, float d1, float d2, float vf0,
                                          float vf1, float vf2, int k, float &ubl, int &ks0,
                                          float &kl0, int &ks1, float &kl1, bool &ovf) {
  const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
  if (dd > Z.near2) return;
  const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
  const float disc = Z.sig2f - (dd - dv * dv);
  if (!(dv < Z.eps_v && disc > -Z.eps_d)) return;
  if (dv < -Z.eps_v && disc > Z.eps_d)
    ubl = fminf(ubl, fmaxf(0.f, -dv + Z.eps_v - sqrt_lo(disc - Z.eps_d)) + 1e-6f);
  const float lb = -dv - Z.eps_v - sqrt_hi(disc + Z.eps_d);
  if (lb > ubl) return;
  const float INF = __int_as_float(0x7f800000);
  if (kl0 > ubl) {
    ks0 = -1;
    kl0 = INF;
  }
  if (kl1 > ubl) {
    ks1 = -1;
    kl1 = INF;
  }
  if (ks0 < 0) {
    ks0 = k;
    kl0 = lb;
  } else if (ks1 < 0) {
    ks1 = k;
    kl1 = lb;
  } else {
    ovf = true;
  }
}

__device__ __forceinline__ float screen_lb(const Screen &Z, float d0, float d1, float d2,
                                           float vf0, float vf1, float vf2, bool &possible) {
  const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
  const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
  const float disc = Z.sig2f - (dd - dv * dv);
  possible = dd <= Z.near2 && dv < Z.eps_v && disc > -Z.eps_d;
  return -dv - Z.eps_v - sqrt_hi(fmaxf(disc + Z.eps_d, 0.f));
}

// Screen the beads of one local cell (16 bytes: count, then up to 6 slots,
// read at once) two per round, so that their shadow loads overlap.  The set
// of candidates a lane keeps or flags does not depend on the order in which
// it screens them (see screen_hs).
__device__ __forceinline__ void screen_cell(const Screen &Z, const Stage &st, const unsigned short *rec,
                                            int p, float a0, float a1, float a2, float w0, float w1,
                                            float w2, float &ubl, int &ks0, float &kl0, int &ks1,
                                            float &kl1, bool &ovf) {
  const uint4 c = *reinterpret_cast<const uint4 *>(rec);
  const int n = (int)c.x;
  const int sl[6] = {(int)(c.y & 0xFFFF), (int)(c.y >> 16), (int)(c.z & 0xFFFF),
                     (int)(c.z >> 16), (int)(c.w & 0xFFFF), (int)(c.w >> 16)};
#pragma unroll
  for (int i = 0; i < 6; i += 2) {
    if (i >= n) break;
    const int ka = sl[i];
    const bool two = i + 1 < n;
    const int kb = two ? sl[i + 1] : ka;
    const float ax = st.fx[ka], ay = st.fy[ka], az = st.fz[ka];
    const float bx = st.fx[kb], by = st.fy[kb], bz = st.fz[kb];
    if (ka != p) screen_hs(Z, a0 - ax, a1 - ay, a2 - az, w0, w1, w2, ka, ubl, ks0, kl0, ks1, kl1, ovf);
    if (two && kb != p)
      screen_hs(Z, a0 - bx, a1 - by, a2 - bz, w0, w1, w2, kb, ubl, ks0, kl0, ks1, kl1, ovf);
  }
}

// FP64 position of staged slot k: shared memory for the first M slots,
// otherwise (a joint bead, static this sweep) the global position array
__device__ __forceinline__ void pos64(const Stage &st, const double *r, int k, bool in_smem,
                                      double &x, double &y, double &z) {
#ifdef ECMC_CHECKED
  x = y = z = 0.0;
  if (st.status && !CHK(k, st.cap, 1, st.status)) return;
  if (!in_smem && st.status && !CHK(st.id[k], st.nglob, 2, st.status)) return;
#endif
  if (in_smem) {
    x = st.px[k];
    y = st.py[k];
    z = st.pz[k];
  } else {
    const int64_t b = st.id[k];
    x = r[3 * b];
    y = r[3 * b + 1];
    z = r[3 * b + 2];
  }
}

// ---------------------------------------------------------------- staging
// Stage one tile (domain) or the whole system (serial) into the group's
// shared memory: the lanes in `mask` call this together (the whole warp, or
// one group of G lanes while the warp's other groups do something else).  Returns the motile count m, the
// hard-sphere joint count j1 and the staged count ns; clears `live` when the
// tile does not fit its capacity.
#define SYS(f) (BATCH ? rp->f : P.f)
template <int G, bool F32, bool BATCH>
__device__ __forceinline__ void stage_tile(const ECParams &P, const RepParams *rp, const Stage &st,
                                           int gl, bool &live, int unit, double c0, double c1,
                                           double c2, double *Rr, const int32_t *Rstart, int S,
                                           int M64, int MNB, int NC, const LGrid &LG, int &m,
                                           int &j1, int &ns, unsigned mask = FULL,
                                           bool *overflow = nullptr) {
  // a tile that does not fit its capacities sets the device status, or, when
  // the caller passes `overflow`, only that flag (the caller stages the tile
  // again later with larger capacities)
  auto capacity = [&]() {
    if (overflow) *overflow = true;
    else if (gl == 0) set_status(P.status, DEV_CAPACITY);
  };
  if (overflow) *overflow = false;
  if (gl == 0) {
    st.hdr[0] = 0;
    st.hdr[1] = 0;
    st.hdr[2] = 0;
    st.hdr[3] = 0;
    st.hdr[4] = 0;
    st.hdr[5] = 0;
    st.hdr[6] = 0;
  }
  __syncwarp(mask);
  m = 0;
  j1 = 0;
  ns = 0;
  if (!P.domain) {
    // serial: every bead, slot = id, all motile
    const int n = (int)P.n;
    for (int b = gl; b < n; b += G) {
      const double x = Rr[3 * (int64_t)b], y = Rr[3 * (int64_t)b + 1], z = Rr[3 * (int64_t)b + 2];
      st.px[b] = x;
      st.py[b] = y;
      st.pz[b] = z;
      st.fx[b] = (float)x;
      st.fy[b] = (float)y;
      st.fz[b] = (float)z;
      st.id[b] = b;
      const int c = b % SYS(N);
      st.nb[b] = nb_pack(c == 0 ? -1 : b - 1, c == SYS(N) - 1 ? -1 : b + 1);
    }
    m = n;
    j1 = 0;
    ns = n;
  } else {
    const double corner[3] = {c0, c1, c2};
    // cell window covering the tether halo of the tile
    int c_lo[3], c_n[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lo = corner[a] - P.halo_te, hi = corner[a] + SYS(W)[a] + P.halo_te;
      int l = (int)floor(lo / SYS(cs)[a]);
      const int h = (int)floor(hi / SYS(cs)[a]);
      int cnt = h - l + 1;
      if (cnt >= SYS(nc)[a]) {
        l = 0;
        cnt = SYS(nc)[a];
      }
      c_lo[a] = l;
      c_n[a] = live ? cnt : 0;
    }
    // pass 1: collect (cell-order index, category|id); the shadow arrays
    // (12 B per slot) serve as 8 B per slot of scratch until pass 3.  The
    // cells of one row of the window (consecutive x) are one contiguous
    // range of the cell-ordered arrays (two when the row wraps around the
    // box); each lane takes whole rows and loads four beads at a time.
    int2 *scr = (int2 *)st.fx;
    // halo membership in FP32 from FP32 copies of the positions, widened by
    // 1e-3 sigma plus four FP32 ulps of the box: a superset of the exact
    // sets (an extra obstacle beyond reach is never hit; a bond partner is
    // always within the tether halo)
    float cf[3], Lf[3], Lhf[3], Wf[3];
    float Lmax = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cf[a] = (float)corner[a];
      Lf[a] = (float)SYS(L)[a];
      Lhf[a] = 0.5f * Lf[a];
      Wf[a] = (float)SYS(W)[a];
      Lmax = fmaxf(Lmax, Lf[a]);
    }
    const float widen = 1e-3f * (float)P.sigma + 4.8e-7f * Lmax;
    const float hs_f = (float)P.halo_hs + widen, te_f = (float)P.halo_te + widen;
    const int nc0 = SYS(nc)[0], nc1 = SYS(nc)[1], nc2 = SYS(nc)[2];
    const int nrows = c_n[1] * c_n[2];
    int cx = c_lo[0] % nc0;
    if (cx < 0) cx += nc0;
    const int len0 = c_n[0] < nc0 - cx ? c_n[0] : nc0 - cx;
    for (int r = gl; r < nrows; r += G) {
      const int qy = r % c_n[1], qz = r / c_n[1];
      int cy = (c_lo[1] + qy) % nc1;
      int cz = (c_lo[2] + qz) % nc2;
      if (cy < 0) cy += nc1;
      if (cz < 0) cz += nc2;
      const int base = (cz * nc1 + cy) * nc0;
      const int a0 = Rstart[base + cx], b0 = Rstart[base + cx + len0];
      int a1 = 0, b1 = 0;
      if (len0 < c_n[0]) {
        a1 = Rstart[base];
        b1 = Rstart[base + c_n[0] - len0];
      }
      const int n0 = b0 - a0, nt = n0 + (b1 - a1);
      for (int k0 = 0; k0 < nt; k0 += 4) {
        int tg[4], jj[4], idv[4];
        float px[4], py[4], pz[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = k0 + u;
          jj[u] = k < n0 ? a0 + k : a1 + (k - n0);
          tg[u] = -2;
          idv[u] = 0;
          px[u] = py[u] = pz[u] = 0.f;
          if (k < nt) {
            const int64_t j = jj[u];
            tg[u] = P.ctag[j];
            idv[u] = P.cid[j];
            px[u] = P.crf[3 * j];
            py[u] = P.crf[3 * j + 1];
            pz[u] = P.crf[3 * j + 2];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (tg[u] == -2) continue;
          int cat = -1;
          if (tg[u] == unit) {
            cat = 0;
          } else if (tg[u] < 0) {
            const float pp[3] = {px[u], py[u], pz[u]};
            bool in_hs = true, in_te = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float sa = pp[a] - cf[a];
              sa = sa > Lhf[a] ? sa - Lf[a] : (sa < -Lhf[a] ? sa + Lf[a] : sa);
              in_hs = in_hs && (sa >= -hs_f) && (sa <= Wf[a] + hs_f);
              in_te = in_te && (sa >= -te_f) && (sa <= Wf[a] + te_f);
            }
            cat = in_hs ? 1 : (in_te ? 2 : -1);
          }
          if (cat >= 0) {
            const int slot = atomicAdd(&st.hdr[2], 1);
            if (slot < S) scr[slot] = make_int2(jj[u], (cat << 29) | idv[u]);
            else st.hdr[3] = 1;
            if (cat < 2) atomicAdd(&st.hdr[5 + cat], 1);
          }
        }
      }
    }
    __syncwarp(mask);
    ns = st.hdr[2];
    if (st.hdr[3]) {
      capacity();
      live = false;
      ns = 0;
    }
    const int ns_max = __reduce_max_sync(mask, ns);
    // pass 2: slots.  Motile beads take their rank by id (the start bead of
    // an EC is the u-th motile bead in id order); joint beads take the next
    // free slot of their category (their order matters to nothing).
    m = st.hdr[5];
    j1 = st.hdr[6];
    for (int s0 = 0; s0 < ns_max; s0 += G) {
      const int s = s0 + gl;
      if (s < ns) {
        const int2 e = scr[s];
        const int cat = e.y >> 29;
        int rank;
        if (cat == 0) {
          rank = 0;
          for (int t = 0; t < ns; ++t) rank += (scr[t].y < e.y);
        } else {
          rank = (cat == 1 ? m : m + j1) + atomicAdd(&st.hdr[cat - 1], 1);
        }
        const int j = e.x;
        if (!CHK(rank, S, 3, P.status)) continue;
        if (rank < M64) {
          st.px[rank] = P.cr[3 * (int64_t)j];
          st.py[rank] = P.cr[3 * (int64_t)j + 1];
          st.pz[rank] = P.cr[3 * (int64_t)j + 2];
        }
        st.id[rank] = e.y & ((1 << 29) - 1);
      }
    }
    __syncwarp(mask);
    if (m > MNB) {  // more motile beads than the motile capacity
      if (live) capacity();
      live = false;
    }
    // pass 2b (bead springs): a spring has no longest bond, so the bonded
    // beads of motile beads are staged wherever they are; one outside the
    // tether halo (a joint bead, static this sweep) is appended after the
    // staged beads (two motile beads may append the same bead twice; both
    // copies are read-only and equal)
    // (the condition is the same for every lane in `mask`: the groups of a
    // warp may hold live and dead tiles, and all of them reach the barrier)
    if (P.k_spring > 0.0) {
      const int Nc = SYS(N);
      for (int s = gl; live && s < m; s += G) {
        const int id = st.id[s];
        const int c = id % Nc;
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
          const int q = dir == 0 ? (c != 0 ? id - 1 : -1) : (c != Nc - 1 ? id + 1 : -1);
          if (q < 0) continue;
          if (!CHK(q, BATCH ? rp->n_beads : P.n, 4, P.status)) continue;
          if (find_id(st.id, 0, m, q) >= 0 || find_id_lin(st.id, m, ns, q) >= 0) continue;
          const int slot = atomicAdd(&st.hdr[2], 1);
          if (slot < S) {
            st.id[slot] = q;
            if (slot < M64) {
              st.px[slot] = Rr[3 * (int64_t)q];
              st.py[slot] = Rr[3 * (int64_t)q + 1];
              st.pz[slot] = Rr[3 * (int64_t)q + 2];
            }
          } else {
            st.hdr[3] = 1;
          }
        }
      }
      __syncwarp(mask);
      if (live) {
        if (st.hdr[3]) {
          capacity();
          live = false;
          ns = 0;
        } else {
          ns = st.hdr[2];
        }
      }
    }
    const int ns_max2 = __reduce_max_sync(mask, ns);
    // pass 3: shadows (FP32 position minus FP32 corner, the form the moved
    // pivot's shadow takes too) and bond partners of motile beads; empty
    // cells.  Four slots at a time (independent loads).
    for (int i = gl; i < NC; i += G) cell_count(st.cell + 8 * i) = 0u;
    const float *Rf = P.rf + (BATCH ? 3 * rp->bead_off : 0);
    for (int s0 = 0; s0 < ns_max2; s0 += 4 * G) {
      float x[4], y[4], z[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int s = s0 + u * G + gl;
        x[u] = y[u] = z[u] = 0.f;
        if (s < ns && live && CHK(st.id[s], BATCH ? rp->n_beads : P.n, 5, P.status)) {
          const int64_t b = st.id[s];
          x[u] = Rf[3 * b];
          y[u] = Rf[3 * b + 1];
          z[u] = Rf[3 * b + 2];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int s = s0 + u * G + gl;
        if (!(s < ns && live)) continue;
        float f0 = x[u] - cf[0], f1 = y[u] - cf[1], f2 = z[u] - cf[2];
        f0 = f0 > Lhf[0] ? f0 - Lf[0] : (f0 < -Lhf[0] ? f0 + Lf[0] : f0);
        f1 = f1 > Lhf[1] ? f1 - Lf[1] : (f1 < -Lhf[1] ? f1 + Lf[1] : f1);
        f2 = f2 > Lhf[2] ? f2 - Lf[2] : (f2 < -Lhf[2] ? f2 + Lf[2] : f2);
        st.fx[s] = f0;
        st.fy[s] = f1;
        st.fz[s] = f2;
        int prev = -1, next = -1;
        if (s < m) {
          const int id = st.id[s];
          const int c = id % SYS(N);
          if (c != 0) {
            prev = find_id(st.id, 0, m, id - 1);
            if (prev < 0) prev = find_id_lin(st.id, m, ns, id - 1);
            if (prev < 0) set_status(P.status, DEV_TILE);
          }
          if (c != SYS(N) - 1) {
            next = find_id(st.id, 0, m, id + 1);
            if (next < 0) next = find_id_lin(st.id, m, ns, id + 1);
            if (next < 0) set_status(P.status, DEV_TILE);
          }
        }
        if (s < MNB) st.nb[s] = nb_pack(prev, next);
      }
    }
    __syncwarp(mask);
    // pass 4: the hard-sphere slots into the local grid, all lanes at once
    // (the order inside a cell does not matter to the screen)
    if (live) {
      for (int s = gl; s < m + j1; s += G) {
        int a0, a1, a2;
        unsigned short *c = st.cell + 8 * lcell(LG, st.fx[s], st.fy[s], st.fz[s], a0, a1, a2);
        const unsigned old = atomicAdd(&cell_count(c), 1u);
        if (old < (unsigned)CELL_CAP) {
          c[2 + old] = (unsigned short)s;
        } else {
          const int k = atomicAdd(&st.hdr[4], 1);
          if (k < st.ovf_cap) st.ovf[k] = (unsigned short)s;
          else st.hdr[3] = 1;
        }
      }
    }
    __syncwarp(mask);
    // counts past a cell's capacity went to the overflow list
    for (int i = gl; i < NC; i += G) {
      unsigned &cc = cell_count(st.cell + 8 * i);
      if (cc > (unsigned)CELL_CAP) cc = CELL_CAP;
    }
    __syncwarp(mask);
    if (st.hdr[3]) {
      if (live) capacity();
      live = false;
      if (gl == 0) st.hdr[4] = 0;
    }
  }
  if (!live) m = 0;
}
#undef SYS

}  // namespace
}  // namespace ecmc
