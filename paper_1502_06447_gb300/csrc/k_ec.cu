// Event-chain kernels (arXiv:1502.06447, Sec. II: EC move; Sec. II.B:
// tile-joint decomposition with reflections; Sec. II.D: swap move).
//
// One group of G lanes (G = 32, 16 or 8) runs the ECs of one tile; the
// 32/G groups of a warp advance in lockstep, one event per iteration, so
// every warp instruction of the serial part serves all of them.
//
// Per tile and sweep the group stages into shared memory every bead the
// tile's ECs can touch, sorted into three id-ordered ranges:
//   [0, m)          motile beads of the tile (start beads, pivots)
//   [m, m + j1)     joint beads within the hard-sphere halo (obstacles)
//   [m + j1, ns)    joint beads within the tether halo only (bond partners)
// The start bead of an EC is then slot below(u, m); bond partners are found
// by binary search on the ids.  Positions are the wrapped FP64 coordinates
// of the global state, so every candidate is evaluated with exactly the
// arithmetic of the plain definition.  FP32 shadows (tile-local) feed the
// screened form.
#include <cuda_runtime.h>
#include <float.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BLOCK_THREADS = 128;

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
  const unsigned long long a = __double_as_longlong(x), b = __double_as_longlong(bx);
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

template <int G>
__device__ __forceinline__ int group_max_i(int v) {
  // lockstep bound over the whole warp
  return __reduce_max_sync(FULL, v);
}

struct Stage {
  double *px, *py, *pz;  // FP64 wrapped positions
  float *fx, *fy, *fz;   // FP32 tile-local shadows
  int *id;               // bead ids (sorted within each range)
  int2 *nb;              // bond partner slots of motile beads (-1: none)
  int *hdr;              // [0] m, [1] j1, [2] ns, [3] overflow
};

__device__ __forceinline__ Stage carve(unsigned char *base, int S) {
  Stage s;
  s.px = (double *)base;
  s.py = s.px + S;
  s.pz = s.py + S;
  s.nb = (int2 *)(s.pz + S);
  s.fx = (float *)(s.nb + S);
  s.fy = s.fx + S;
  s.fz = s.fy + S;
  s.id = (int *)(s.fz + S);
  s.hdr = s.id + S;
  return s;
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

__device__ __forceinline__ void set_status(int *st, int code) { atomicCAS(st, 0, code); }

template <int G, bool F32>
__global__ void __launch_bounds__(BLOCK_THREADS) ec_kernel(const ECParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gib = threadIdx.x / G;
  const int gpb = blockDim.x / G;
  const int unit = blockIdx.x * gpb + gib;
  const int S = P.stage_cap;
  const size_t per_group = (size_t)S * 48 + 32;
  Stage st = carve(smem + (size_t)gib * per_group, S);
  bool live = unit < P.n_units;

  // tile geometry (domain) or the whole box (serial)
  int tk[3] = {0, 0, 0};
  double corner[3] = {0.0, 0.0, 0.0};
  if (P.domain && live) {
    tk[0] = unit % P.D[0];
    tk[1] = (unit / P.D[0]) % P.D[1];
    tk[2] = unit / (P.D[0] * P.D[1]);
  }
  // corner = shift + k T (the shift first, then the tile offset)
  if (P.domain && live) {
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)P.sweep, 0, 0, P.seed, P.replica);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double sh = unit53(w.v[a]) * P.T[a];
      corner[a] = sh + (double)tk[a] * P.T[a];
    }
  }

  // ------------------------------------------------------------ staging
  if (gl == 0) {
    st.hdr[0] = 0;
    st.hdr[1] = 0;
    st.hdr[2] = 0;
    st.hdr[3] = 0;
  }
  __syncwarp();
  int m = 0, j1 = 0, ns = 0;
  if (!P.domain) {
    // serial: every bead, slot = id, all motile
    const int n = (int)P.n;
    for (int b = gl; b < n; b += G) {
      const double x = P.r[3 * (int64_t)b], y = P.r[3 * (int64_t)b + 1], z = P.r[3 * (int64_t)b + 2];
      st.px[b] = x;
      st.py[b] = y;
      st.pz[b] = z;
      st.fx[b] = (float)x;
      st.fy[b] = (float)y;
      st.fz[b] = (float)z;
      st.id[b] = b;
      const int c = b % P.N;
      st.nb[b] = make_int2(c == 0 ? -1 : b - 1, c == P.N - 1 ? -1 : b + 1);
    }
    m = n;
    j1 = 0;
    ns = n;
  } else {
    // cell window covering the tether halo of the tile
    int c_lo[3], c_n[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double lo = corner[a] - P.halo_te, hi = corner[a] + P.W[a] + P.halo_te;
      int l = (int)floor(lo / P.cs[a]);
      int h = (int)floor(hi / P.cs[a]);
      int cnt = h - l + 1;
      if (cnt >= P.nc[a]) {
        l = 0;
        cnt = P.nc[a];
      }
      c_lo[a] = l;
      c_n[a] = live ? cnt : 0;
    }
    const int ncell = c_n[0] * c_n[1] * c_n[2];
    const int ncell_max = __reduce_max_sync(FULL, ncell);
    // pass 1: collect (cell-order index, category|id) in the nb scratch
    for (int q0 = 0; q0 < ncell_max; q0 += G) {
      const int q = q0 + gl;
      if (q < ncell) {
        const int qx = q % c_n[0], qy = (q / c_n[0]) % c_n[1], qz = q / (c_n[0] * c_n[1]);
        int cx = (c_lo[0] + qx) % P.nc[0];
        int cy = (c_lo[1] + qy) % P.nc[1];
        int cz = (c_lo[2] + qz) % P.nc[2];
        if (cx < 0) cx += P.nc[0];
        if (cy < 0) cy += P.nc[1];
        if (cz < 0) cz += P.nc[2];
        const int cell = (cz * P.nc[1] + cy) * P.nc[0] + cx;
        const int j0 = P.cstart[cell], jend = P.cstart[cell + 1];
        for (int j = j0; j < jend; ++j) {
          const int tg = P.ctag[j];
          int cat = -1;
          if (tg == unit) {
            cat = 0;
          } else if (tg < 0) {
            bool in_hs = true, in_te = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const double s = wrap_d(P.cr[3 * (int64_t)j + a] - corner[a], P.L[a], P.half[a]);
              in_hs = in_hs && (s >= -P.halo_hs) && (s <= P.W[a] + P.halo_hs);
              in_te = in_te && (s >= -P.halo_te) && (s <= P.W[a] + P.halo_te);
            }
            cat = in_hs ? 1 : (in_te ? 2 : -1);
          }
          if (cat >= 0) {
            const int slot = atomicAdd(&st.hdr[2], 1);
            if (slot < S) st.nb[slot] = make_int2(j, (cat << 29) | P.cid[j]);
            else st.hdr[3] = 1;
          }
        }
      }
    }
    __syncwarp();
    ns = st.hdr[2];
    if (st.hdr[3]) {
      if (gl == 0) set_status(P.status, DEV_CAPACITY);
      live = false;
      ns = 0;
    }
    const int ns_max = __reduce_max_sync(FULL, ns);
    // pass 2: rank by (category, id) and place into the sorted slots
    int cnt_cat0 = 0, cnt_cat1 = 0;
    for (int s0 = 0; s0 < ns_max; s0 += G) {
      const int s = s0 + gl;
      int2 e = make_int2(0, 0);
      int rank = 0;
      if (s < ns) {
        e = st.nb[s];
        for (int t = 0; t < ns; ++t) rank += (st.nb[t].y < e.y);
        const int cat = e.y >> 29;
        cnt_cat0 += (cat == 0);
        cnt_cat1 += (cat == 1);
      }
      __syncwarp();
      if (s < ns) {
        const int j = e.x;
        const double x = P.cr[3 * (int64_t)j], y = P.cr[3 * (int64_t)j + 1], z = P.cr[3 * (int64_t)j + 2];
        st.px[rank] = x;
        st.py[rank] = y;
        st.pz[rank] = z;
        st.fx[rank] = (float)wrap_d(x - corner[0], P.L[0], P.half[0]);
        st.fy[rank] = (float)wrap_d(y - corner[1], P.L[1], P.half[1]);
        st.fz[rank] = (float)wrap_d(z - corner[2], P.L[2], P.half[2]);
        st.id[rank] = e.y & ((1 << 29) - 1);
      }
      __syncwarp();
    }
    // group sums of the category counts
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      cnt_cat0 += __shfl_xor_sync(FULL, cnt_cat0, off);
      cnt_cat1 += __shfl_xor_sync(FULL, cnt_cat1, off);
    }
    m = cnt_cat0;
    j1 = cnt_cat1;
    // pass 3: bond partners of motile beads
    for (int s0 = 0; s0 < ns_max; s0 += G) {
      const int s = s0 + gl;
      if (s < m) {
        const int id = st.id[s];
        const int c = id % P.N;
        int2 nbv = make_int2(-1, -1);
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
          const bool has = dir == 0 ? (c != 0) : (c != P.N - 1);
          if (!has) continue;
          const int want = dir == 0 ? id - 1 : id + 1;
          int f = find_id(st.id, 0, m, want);
          if (f < 0) f = find_id(st.id, m, m + j1, want);
          if (f < 0) f = find_id(st.id, m + j1, ns, want);
          if (f < 0) set_status(P.status, DEV_TILE);
          if (dir == 0) nbv.x = f;
          else nbv.y = f;
        }
        st.nb[s] = nbv;
      }
    }
    __syncwarp();
  }
  if (!live) m = 0;
  const int nhs = m + j1;
  const int nhs_max = __reduce_max_sync(FULL, nhs);

  // ------------------------------------------------------------ ECs
  const int n_ec = P.ecs_per_tile;
  const float sigf = (float)P.sigma;
  const float sig2f = (float)P.sig2;
  const float near2 = (float)((P.s_cap + P.sigma + 0.01 * P.sigma) * (P.s_cap + P.sigma + 0.01 * P.sigma));
  for (int e = 0; e < n_ec; ++e) {
    bool active = live && m > 0;
    // start bead and direction
    const uint64_t c0 = P.domain ? (TAG_START | ((uint64_t)e << 8)) : TAG_START;
    const uint64_t c1 = P.domain ? (uint64_t)P.sweep : 0;
    const uint64_t c2 = P.domain ? (uint64_t)unit : (uint64_t)(P.sweep + e);
    int p = 0;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (active) {
      u64x4 w = philox(c0, c1, c2, 0, P.seed, P.replica);
      p = (int)scale_below(w.v[0], (uint64_t)m);
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
          w = philox(c0, c1, c2, att, P.seed, P.replica);
          a = 2.0 * unit53(w.v[0]) - 1.0;
          b = 2.0 * unit53(w.v[1]) - 1.0;
          c = 2.0 * unit53(w.v[2]) - 1.0;
        }
      }
    }
    int pid = active ? st.id[p] : 0;
    double q0 = active ? st.px[p] : 0.0, q1 = active ? st.py[p] : 0.0, q2 = active ? st.pz[p] : 0.0;
    float pf0 = active ? st.fx[p] : 0.f, pf1 = active ? st.fy[p] : 0.f, pf2 = active ? st.fz[p] : 0.f;
    float vf0 = (float)v0, vf1 = (float)v1, vf2 = (float)v2;
    double xrem = P.ell;
    int64_t nev = 0;
    int64_t ncontact = 0;
    u64x4 swr;
    swr.v[0] = swr.v[1] = swr.v[2] = swr.v[3] = 0;
    uint64_t h = 0xCBF29CE484222325ull;
    double lift = 0.0, refl = 0.0, disp = 0.0;
    unsigned long long cnt[ECMC_NEV];
#pragma unroll
    for (int k = 0; k < ECMC_NEV; ++k) cnt[k] = 0;
    unsigned long long tried = 0;
    unsigned long long confirmed = 0;

    while (__any_sync(FULL, active)) {
      if (active && nev >= P.event_cap) {
        if (gl == 0) set_status(P.status, DEV_STUCK);
        active = false;
      }
      // special candidates, one per lane: end/pass, two tethers, three walls
      double bx = __longlong_as_double(0x7ff0000000000000ll);  // +inf
      uint64_t bkey = ~0ull;
      if (active) {
        if (gl == 0) {
          if (P.s_cap < xrem) {
            bx = P.s_cap;
            bkey = make_key(KIND_PASS, 0, 0);
          } else {
            bx = xrem;
            bkey = make_key(KIND_END, 0, 0);
          }
        } else if (gl <= 2) {
          const int2 nbv = st.nb[p];
          const int t = gl == 1 ? nbv.x : nbv.y;
          if (t >= 0) {
            const double d0 = wrap_d(q0 - st.px[t], P.L[0], P.half[0]);
            const double d1 = wrap_d(q1 - st.py[t], P.L[1], P.half[1]);
            const double d2 = wrap_d(q2 - st.pz[t], P.L[2], P.half[2]);
            bx = tether_x(d0, d1, d2, v0, v1, v2, P.b2);
            bkey = make_key(KIND_TETHER, st.id[t], t);
          }
        } else if (gl <= 5 && P.domain) {
          const int a = gl - 3;
          const double va = a == 0 ? v0 : (a == 1 ? v1 : v2);
          const double qa = a == 0 ? q0 : (a == 1 ? q1 : q2);
          if (va != 0.0) {
            const double loc = wrap_d(qa - corner[a], P.L[a], P.half[a]);
            double x = va > 0.0 ? (P.W[a] - loc) / va : (0.0 - loc) / va;
            if (x < 0.0) x = 0.0;
            bx = x;
            bkey = make_key(KIND_WALL, a, 0);
          }
        }
      }
      if (!F32) {
        // plain FP64: every staged obstacle is a candidate
        for (int k0 = 0; k0 < nhs_max; k0 += G) {
          const int k = k0 + gl;
          if (active && k < nhs && k != p) {
            const double d0 = wrap_d(q0 - st.px[k], P.L[0], P.half[0]);
            const double d1 = wrap_d(q1 - st.py[k], P.L[1], P.half[1]);
            const double d2 = wrap_d(q2 - st.pz[k], P.L[2], P.half[2]);
            const double x = contact_x(d0, d1, d2, v0, v1, v2, P.sig2);
            if (x >= 0.0) {
              const uint64_t key = make_key(KIND_HS, st.id[k], k);
              if (better(x, key, bx, bkey)) {
                bx = x;
                bkey = key;
              }
            }
          }
        }
      } else {
        // FP32 screen: U bounds the smallest candidate from above; only
        // beads whose lower bound |d| - sigma can reach U are confirmed in
        // FP64 (the margins cover the FP32 rounding of tile-local coordinates)
        float ub = __double2float_ru(bx);
        for (int k0 = 0; k0 < nhs_max; k0 += G) {
          const int k = k0 + gl;
          if (active && k < nhs && k != p) {
            float d0 = pf0 - st.fx[k], d1 = pf1 - st.fy[k], d2 = pf2 - st.fz[k];
            if (!P.domain) {
              d0 = d0 > 0.5f * (float)P.L[0] ? d0 - (float)P.L[0] : (d0 < -0.5f * (float)P.L[0] ? d0 + (float)P.L[0] : d0);
              d1 = d1 > 0.5f * (float)P.L[1] ? d1 - (float)P.L[1] : (d1 < -0.5f * (float)P.L[1] ? d1 + (float)P.L[1] : d1);
              d2 = d2 > 0.5f * (float)P.L[2] ? d2 - (float)P.L[2] : (d2 < -0.5f * (float)P.L[2] ? d2 + (float)P.L[2] : d2);
            }
            const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
            if (dd <= near2) {
              const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
              const float disc = sig2f - (dd - dv * dv);
              if (dv < -P.eps_v && disc > P.eps_d) {
                const float u = fmaxf(0.f, -dv - sqrtf(disc - P.eps_d)) + P.eps_x;
                ub = fminf(ub, u);
              }
            }
          }
        }
        const float U = group_minf<G>(ub);
        const float rr = U + sigf + P.eps_x;
        const float lb2 = rr * rr * 1.000001f;
        for (int k0 = 0; k0 < nhs_max; k0 += G) {
          const int k = k0 + gl;
          if (active && k < nhs && k != p) {
            float d0 = pf0 - st.fx[k], d1 = pf1 - st.fy[k], d2 = pf2 - st.fz[k];
            if (!P.domain) {
              d0 = d0 > 0.5f * (float)P.L[0] ? d0 - (float)P.L[0] : (d0 < -0.5f * (float)P.L[0] ? d0 + (float)P.L[0] : d0);
              d1 = d1 > 0.5f * (float)P.L[1] ? d1 - (float)P.L[1] : (d1 < -0.5f * (float)P.L[1] ? d1 + (float)P.L[1] : d1);
              d2 = d2 > 0.5f * (float)P.L[2] ? d2 - (float)P.L[2] : (d2 < -0.5f * (float)P.L[2] ? d2 + (float)P.L[2] : d2);
            }
            const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
            if (dd <= lb2) {
              const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
              const float disc = sig2f - (dd - dv * dv);
              if (dv < P.eps_v && disc > -P.eps_d) {
                ++confirmed;
                const double e0 = wrap_d(q0 - st.px[k], P.L[0], P.half[0]);
                const double e1 = wrap_d(q1 - st.py[k], P.L[1], P.half[1]);
                const double e2 = wrap_d(q2 - st.pz[k], P.L[2], P.half[2]);
                const double x = contact_x(e0, e1, e2, v0, v1, v2, P.sig2);
                if (x >= 0.0) {
                  const uint64_t key = make_key(KIND_HS, st.id[k], k);
                  if (better(x, key, bx, bkey)) {
                    bx = x;
                    bkey = key;
                  }
                }
              }
            }
          }
        }
      }
      group_argmin<G>(bx, bkey);
      __syncwarp();

      int np = p;
      if (active) {
        const double x = bx;
        const int kind = key_kind(bkey);
        const int slot = key_slot(bkey);
        const int64_t partner = (kind == KIND_END || kind == KIND_PASS) ? -1 : key_id(bkey);
        // move the pivot
        const int di0 = step_axis(q0, x, v0, P.L[0]);
        const int di1 = step_axis(q1, x, v1, P.L[1]);
        const int di2 = step_axis(q2, x, v2, P.L[2]);
        if (gl == 0) {
          if (di0) P.img[3 * (int64_t)pid] += di0;
          if (di1) P.img[3 * (int64_t)pid + 1] += di1;
          if (di2) P.img[3 * (int64_t)pid + 2] += di2;
        }
        disp = disp + x;
        ++nev;
        int out;
        bool moved_pivot_slot = false;  // pivot's own slot now holds a new position
        if (kind == KIND_END) {
          out = ECMC_EV_END;
        } else if (kind == KIND_PASS) {
          out = ECMC_EV_PASS;
        } else if (kind == KIND_WALL) {
          out = ECMC_EV_WALL;
          if (partner == 0) v0 = -v0;
          else if (partner == 1) v1 = -v1;
          else v2 = -v2;
        } else {
          const double k0 = st.px[slot], k1 = st.py[slot], k2 = st.pz[slot];
          const double d0 = wrap_d(q0 - k0, P.L[0], P.half[0]);
          const double d1 = wrap_d(q1 - k1, P.L[1], P.half[1]);
          const double d2 = wrap_d(q2 - k2, P.L[2], P.half[2]);
          const double proj = 0.0 - (d0 * v0 + d1 * v1 + d2 * v2);
          const bool motile = slot < m;
          if (!motile) {
            out = kind == KIND_HS ? ECMC_EV_HS_REFLECT : ECMC_EV_TE_REFLECT;
            refl = refl + proj;
            mirror(v0, v1, v2, d0, d1, d2);
          } else if (kind == KIND_HS) {
            lift = lift + proj;
            bool swapped = false;
            if (P.p_swap > 0.0) {
              bool go;
              if (P.p_swap >= 1.0) {
                go = true;
              } else {
                if ((ncontact & 3) == 0)
                  swr = philox(TAG_SWAP | ((uint64_t)(P.domain ? e : 0) << 8), c1, c2,
                               (uint64_t)(ncontact >> 2), P.seed, P.replica);
                go = unit53(swr.v[ncontact & 3]) < P.p_swap;
              }
              ++ncontact;
              if (go) {
                ++tried;
                // bonds of the pivot (slot p) and the hit bead (slot) with the
                // two positions exchanged must all stay within b_max
                bool ok = true;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                  const int a = side == 0 ? p : slot;
                  const double a0 = side == 0 ? k0 : q0;  // new position of a
                  const double a1 = side == 0 ? k1 : q1;
                  const double a2 = side == 0 ? k2 : q2;
                  const int2 nbv = st.nb[a];
#pragma unroll
                  for (int dir = 0; dir < 2; ++dir) {
                    const int b = dir == 0 ? nbv.x : nbv.y;
                    if (b < 0) continue;
                    double b0, b1, b2;
                    if (b == p) {
                      b0 = k0; b1 = k1; b2 = k2;
                    } else if (b == slot) {
                      b0 = q0; b1 = q1; b2 = q2;
                    } else {
                      b0 = st.px[b]; b1 = st.py[b]; b2 = st.pz[b];
                    }
                    const double e0 = wrap_d(a0 - b0, P.L[0], P.half[0]);
                    const double e1 = wrap_d(a1 - b1, P.L[1], P.half[1]);
                    const double e2 = wrap_d(a2 - b2, P.L[2], P.half[2]);
                    ok = ok && (e0 * e0 + e1 * e1 + e2 * e2 <= P.b2);
                  }
                }
                if (ok) {
                  swapped = true;
                  // exchange positions and image counters; the pivot stays
                  if (gl == 0) {
                    st.px[slot] = q0;
                    st.py[slot] = q1;
                    st.pz[slot] = q2;
                    const int kid = st.id[slot];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                      const int ti = P.img[3 * (int64_t)pid + a];
                      P.img[3 * (int64_t)pid + a] = P.img[3 * (int64_t)kid + a];
                      P.img[3 * (int64_t)kid + a] = ti;
                    }
                  }
                  moved_pivot_slot = true;
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
#pragma unroll
        for (int k = 0; k < ECMC_NEV; ++k) cnt[k] += (out == k);
        if (gl == 0) {
          fnv_mix(h, (uint64_t)pid);
          fnv_mix(h, ((uint64_t)(uint32_t)out << 32) | (uint64_t)(uint32_t)partner);
          fnv_mix(h, (uint64_t)__double_as_longlong(x));
          if (P.log) {
            const unsigned long long at = atomicAdd(P.log_n, 1ull);
            if ((int64_t)at < P.log_cap) {
              ecmc_event ev;
              ev.unit = P.rec_offset + (P.domain ? (int64_t)unit * n_ec + e : (int64_t)e);
              ev.seq = (int32_t)(nev - 1);
              ev.pivot = pid;
              ev.kind = out;
              ev.pad = 0;
              ev.partner = partner;
              ev.x = x;
              P.log[at] = ev;
            }
          }
        }
        // store the pivot's (possibly swapped) position and its FP32 shadow
        if (gl == 0) {
          st.px[p] = q0;
          st.py[p] = q1;
          st.pz[p] = q2;
        }
        if (F32) {
          float nf0, nf1, nf2;
          if (P.domain) {
            nf0 = (float)wrap_d(q0 - corner[0], P.L[0], P.half[0]);
            nf1 = (float)wrap_d(q1 - corner[1], P.L[1], P.half[1]);
            nf2 = (float)wrap_d(q2 - corner[2], P.L[2], P.half[2]);
          } else {
            nf0 = (float)q0;
            nf1 = (float)q1;
            nf2 = (float)q2;
          }
          if (gl == 0) {
            st.fx[p] = nf0;
            st.fy[p] = nf1;
            st.fz[p] = nf2;
            if (moved_pivot_slot) {
              // the hit bead now sits at the pivot's old contact position
              const double o0 = st.px[slot], o1 = st.py[slot], o2 = st.pz[slot];
              if (P.domain) {
                st.fx[slot] = (float)wrap_d(o0 - corner[0], P.L[0], P.half[0]);
                st.fy[slot] = (float)wrap_d(o1 - corner[1], P.L[1], P.half[1]);
                st.fz[slot] = (float)wrap_d(o2 - corner[2], P.L[2], P.half[2]);
              } else {
                st.fx[slot] = (float)o0;
                st.fy[slot] = (float)o1;
                st.fz[slot] = (float)o2;
              }
            }
          }
          pf0 = nf0;
          pf1 = nf1;
          pf2 = nf2;
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
        }
      }
      __syncwarp();
      // hand the chain to the new pivot (after the stores above)
      if (active && np != p) {
        p = np;
        pid = st.id[p];
        q0 = st.px[p];
        q1 = st.py[p];
        q2 = st.pz[p];
        if (F32) {
          pf0 = st.fx[p];
          pf1 = st.fy[p];
          pf2 = st.fz[p];
        }
      }
      __syncwarp();
    }
    // EC bookkeeping
    if (F32) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) confirmed += __shfl_xor_sync(FULL, confirmed, off);
    }
    if (live && m > 0 && gl == 0) {
      if (confirmed) atomicAdd(&P.counters[CNT_CONFIRMED], confirmed);
      for (int k = 0; k < ECMC_NEV; ++k)
        if (cnt[k]) atomicAdd(&P.counters[k], cnt[k]);
      atomicAdd(&P.counters[CNT_EVENTS], (unsigned long long)nev);
      if (tried) atomicAdd(&P.counters[CNT_SWAP_TRIED], tried);
      atomicAdd(&P.counters[CNT_ECS], 1ull);
      atomicAdd(&P.sums[SUM_LIFT], lift);
      atomicAdd(&P.sums[SUM_REFL], refl);
      atomicAdd(&P.sums[SUM_DISP], disp);
      if (P.rec_digest) {
        const int64_t idx = P.rec_offset + (P.domain ? (int64_t)unit * n_ec + e : (int64_t)e);
        if (idx < P.rec_cap) {
          P.rec_digest[idx] = h;
          P.rec_lift[idx] = lift;
          P.rec_events[idx] = nev;
        }
      }
    }
    __syncwarp();
  }

  // ------------------------------------------------------------ write back
  if (live) {
    for (int s = gl; s < m; s += G) {
      const int64_t b = st.id[s];
      P.r[3 * b] = st.px[s];
      P.r[3 * b + 1] = st.py[s];
      P.r[3 * b + 2] = st.pz[s];
    }
  }
}

}  // namespace
}  // namespace ecmc

namespace ecmc {

size_t ec_smem_bytes(int stage_cap, int lanes, int groups_per_block) {
  (void)lanes;
  return (size_t)groups_per_block * ((size_t)stage_cap * 48 + 32);
}

template <int G, bool F32>
static cudaError_t launch_t(const ECParams &P, cudaStream_t s) {
  static int smem_max = 0;
  if (!smem_max) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
  }
  // whole warps per block (lockstep shuffles use all 32 lanes), at most 128
  // threads, and the staging buffers of all groups within shared memory
  const int per_warp = 32 / G;
  const size_t per_group = ec_smem_bytes(P.stage_cap, G, 1);
  int gpb = 128 / G;
  while (gpb > per_warp && (size_t)gpb * per_group > (size_t)smem_max) gpb -= per_warp;
  const int need = (P.n_units + per_warp - 1) / per_warp * per_warp;
  if (gpb > need) gpb = need;
  if ((size_t)gpb * per_group > (size_t)smem_max) return cudaErrorInvalidValue;
  const int threads = gpb * G;
  const size_t smem = (size_t)gpb * per_group;
  cudaError_t e = cudaFuncSetAttribute(ec_kernel<G, F32>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (P.n_units + gpb - 1) / gpb;
  ec_kernel<G, F32><<<blocks, threads, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_ec(const ECParams &P, int lanes, int fp32f, cudaStream_t s) {
  if (lanes == 32) return fp32f ? launch_t<32, true>(P, s) : launch_t<32, false>(P, s);
  if (lanes == 16) return fp32f ? launch_t<16, true>(P, s) : launch_t<16, false>(P, s);
  if (lanes == 8) return fp32f ? launch_t<8, true>(P, s) : launch_t<8, false>(P, s);
  return cudaErrorInvalidValue;
}

}  // namespace ecmc
