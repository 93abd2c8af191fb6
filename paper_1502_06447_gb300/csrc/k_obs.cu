// Fused observables over the current state and the initial lattice.
//
//   R_e^2 per chain from minimum-image bonds (end-to-end distance, Sec. IV
//   and the ideal-chain law <R^2> = c N sigma^2); bond lengths and tether
//   violations (b > b_max); hard-sphere overlaps (Eq. 1) from the cell list;
//   g1, the mean-square displacement of the middle bead N/2 (Eq. for g1 in
//   Sec. IV) against a reference snapshot of unwrapped positions; pair and
//   bond counts in thin shells at contact (sigma, b_max) for the
//   contact-value pressure.
#include <cuda_runtime.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

__device__ __forceinline__ void atomic_max_pos(double *a, double v) {
  atomicMax((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_pos(double *a, double v) {
  atomicMin((unsigned long long *)a, (unsigned long long)__double_as_longlong(v));
}

// out_d: [0] sum R_e^2, [1] max bond, [2] min bond, [3] sum g1, [4] sum of bond lengths
// out_u: [0] overlaps, [1] tether violations, [4] [5] bonds in the shells
// (t1, t0] and (t2, t1] below b_max
__global__ void k_chains(const ObsParams O) {
  const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nch = O.n / O.N;
  if (ch >= nch) return;
  double R0 = 0.0, R1 = 0.0, R2 = 0.0, bmax = 0.0, bmin = 1e300, bsum = 0.0;
  unsigned long long viol = 0, tb0 = 0, tb1 = 0;
  const double lim = O.b2 * (1.0 + 1e-10);
  for (int j = 0; j + 1 < O.N; ++j) {
    const int64_t b = ch * O.N + j;
    const double d0 = wrap_d(O.r[3 * (b + 1)] - O.r[3 * b], O.L[0], O.half[0]);
    const double d1 = wrap_d(O.r[3 * (b + 1) + 1] - O.r[3 * b + 1], O.L[1], O.half[1]);
    const double d2 = wrap_d(O.r[3 * (b + 1) + 2] - O.r[3 * b + 2], O.L[2], O.half[2]);
    R0 += d0;
    R1 += d1;
    R2 += d2;
    const double dd = d0 * d0 + d1 * d1 + d2 * d2;
    viol += dd > lim;
    tb0 += (dd > O.c_t1 && dd <= O.c_t0);
    tb1 += (dd > O.c_t2 && dd <= O.c_t1);
    const double bl = sqrt(dd);
    bmax = fmax(bmax, bl);
    bmin = fmin(bmin, bl);
    bsum += bl;
  }
  atomicAdd(&O.out_d[0], R0 * R0 + R1 * R1 + R2 * R2);
  if (O.N > 1) {
    atomicAdd(&O.out_d[4], bsum);
    atomic_max_pos(&O.out_d[1], bmax);
    atomic_min_pos(&O.out_d[2], bmin);
  }
  if (viol) atomicAdd(&O.out_u[1], viol);
  if (tb0) atomicAdd(&O.out_u[4], tb0);
  if (tb1) atomicAdd(&O.out_u[5], tb1);
  if (O.g1ref) {
    const int64_t b = ch * O.N + O.N / 2;
    double g = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double u = O.r[3 * b + a] + (double)O.img[3 * b + a] * O.L[a];
      const double d = u - O.g1ref[3 * ch + a];
      g += d * d;
    }
    atomicAdd(&O.out_d[3], g);
  }
}

__global__ void k_snapshot(const ObsParams O, double *ref) {
  const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nch = O.n / O.N;
  if (ch >= nch) return;
  const int64_t b = ch * O.N + O.N / 2;
#pragma unroll
  for (int a = 0; a < 3; ++a) ref[3 * ch + a] = O.r[3 * b + a] + (double)O.img[3 * b + a] * O.L[a];
}

// pairs i < j closer than sigma (1 - 1e-10)^(1/2), and pairs in the shells
// [lo, s1) and [s1, s2) above sigma, through the cell list (cell side >=
// sqrt(s2), at least 3 cells per axis)
__global__ void k_overlaps(const ObsParams O) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= O.n) return;
  const int c = O.cell[i];
  const int cx = c % O.nc[0], cy = (c / O.nc[0]) % O.nc[1], cz = c / (O.nc[0] * O.nc[1]);
  const double p0 = O.r[3 * i], p1 = O.r[3 * i + 1], p2 = O.r[3 * i + 2];
  const double lim = O.sig2 * (1.0 - 1e-10);
  unsigned long long cnt = 0, cs0 = 0, cs1 = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = (cx + dx + O.nc[0]) % O.nc[0];
        const int y = (cy + dy + O.nc[1]) % O.nc[1];
        const int z = (cz + dz + O.nc[2]) % O.nc[2];
        const int cc = (z * O.nc[1] + y) * O.nc[0] + x;
        for (int j = O.cstart[cc]; j < O.cstart[cc + 1]; ++j) {
          if (O.cid[j] <= i) continue;
          const double d0 = wrap_d(p0 - O.cr[3 * (int64_t)j], O.L[0], O.half[0]);
          const double d1 = wrap_d(p1 - O.cr[3 * (int64_t)j + 1], O.L[1], O.half[1]);
          const double d2 = wrap_d(p2 - O.cr[3 * (int64_t)j + 2], O.L[2], O.half[2]);
          const double dd = d0 * d0 + d1 * d1 + d2 * d2;
          cnt += dd < lim;
          cs0 += (dd >= O.c_lo && dd < O.c_s1);
          cs1 += (dd >= O.c_s1 && dd < O.c_s2);
        }
      }
  if (cnt) atomicAdd(&O.out_u[0], cnt);
  if (cs0) atomicAdd(&O.out_u[2], cs0);
  if (cs1) atomicAdd(&O.out_u[3], cs1);
}

__global__ void k_lattice(int n0, int n1, int n2, double a, double jitter, uint64_t seed,
                          uint64_t replica, double *r, int64_t n) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int64_t plane = (int64_t)n0 * n1;
  const int z = (int)(b / plane);
  const int64_t rem = b % plane;
  const int yy = (int)(rem / n0), xx = (int)(rem % n0);
  const int y = (z % 2 == 0) ? yy : n1 - 1 - yy;
  const int row = z * n1 + yy;
  const int x = (row % 2 == 0) ? xx : n0 - 1 - xx;
  const int site[3] = {x, y, z};
  u64x4 w;
  w.v[0] = w.v[1] = w.v[2] = w.v[3] = 0;
  if (jitter != 0.0) w = philox(TAG_JITTER, 0, (uint64_t)b, 0, seed, replica);
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double p = ((double)site[ax] + 0.5) * a;
    if (jitter != 0.0) p = p + jitter * (2.0 * unit53(w.v[ax]) - 1.0);
    r[3 * b + ax] = p;
  }
}

// beads that overlap another bead (|d|^2 < thr, minimum image, squared
// length (d0 d0 + d1 d1) + d2 d2) through the cell list: flag 0/1 per bead
// and their number (the push-off's start beads, Sec. II.B)
__global__ void k_po_flags(const ObsParams O, double thr, uint8_t *flag, unsigned long long *count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= O.n) return;
  const int c = O.cell[i];
  const int cx = c % O.nc[0], cy = (c / O.nc[0]) % O.nc[1], cz = c / (O.nc[0] * O.nc[1]);
  const double p0 = O.r[3 * i], p1 = O.r[3 * i + 1], p2 = O.r[3 * i + 2];
  uint8_t f = 0;
  for (int dz = -1; dz <= 1 && !f; ++dz)
    for (int dy = -1; dy <= 1 && !f; ++dy)
      for (int dx = -1; dx <= 1 && !f; ++dx) {
        const int x = (cx + dx + O.nc[0]) % O.nc[0];
        const int y = (cy + dy + O.nc[1]) % O.nc[1];
        const int z = (cz + dz + O.nc[2]) % O.nc[2];
        const int cc = (z * O.nc[1] + y) * O.nc[0] + x;
        for (int j = O.cstart[cc]; j < O.cstart[cc + 1]; ++j) {
          if (O.cid[j] == i) continue;
          const double d0 = wrap_d(p0 - O.cr[3 * (int64_t)j], O.L[0], O.half[0]);
          const double d1 = wrap_d(p1 - O.cr[3 * (int64_t)j + 1], O.L[1], O.half[1]);
          const double d2 = wrap_d(p2 - O.cr[3 * (int64_t)j + 2], O.L[2], O.half[2]);
          if ((d0 * d0 + d1 * d1) + d2 * d2 < thr) {
            f = 1;
            break;
          }
        }
      }
  flag[i] = f;
  if (f) atomicAdd(count, 1ull);
}

// Phantom chains (Sec. II.B, first stage of the initial configuration):
// one thread per chain walks N beads with bond length `bond`, the first bead
// uniform in the box, the first bond uniform on the sphere, every next bond
// uniform on the cap t_j . t_{j+1} >= ct around the one before (cos theta =
// 1 - u (1 - ct); the azimuth from the first point of the unit disc drawn
// as (2u - 1, 2u' - 1), at most 256 attempts; the orthonormal pair of t_j
// after Duff et al., "Building an orthonormal basis, revisited", JCGT 2017);
// Philox4x64-10 key (seed, 0), counter (TAG_PHANTOM, chain, bead, attempt).
// Writes unwrapped positions; launch_wrap folds them into the box.
__global__ void k_phantom(int64_t nch, int N, double L0, double L1, double L2, double bond,
                          double ct, uint64_t seed, double *r, unsigned long long *bad) {
  const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (ch >= nch) return;
  u64x4 w = philox(TAG_PHANTOM, (uint64_t)ch, 0, 0, seed, 0);
  double p0 = unit53(w.v[0]) * L0, p1 = unit53(w.v[1]) * L1, p2 = unit53(w.v[2]) * L2;
  double t0 = 0.0, t1 = 0.0, t2 = 1.0;
  double *rc = r + 3 * ch * N;
  rc[0] = p0;
  rc[1] = p1;
  rc[2] = p2;
  for (int j = 1; j < N; ++j) {
    const double ctj = j == 1 ? -1.0 : ct;
    w = philox(TAG_PHANTOM, (uint64_t)ch, (uint64_t)j, 0, seed, 0);
    const double cth = 1.0 - unit53(w.v[0]) * (1.0 - ctj);
    double x = 2.0 * unit53(w.v[1]) - 1.0, y = 2.0 * unit53(w.v[2]) - 1.0;
    double s = x * x + y * y;
    for (uint64_t att = 1; !(s > 0.0 && s <= 1.0); ++att) {
      if (att == 256) {
        atomicAdd(bad, 1ull);
        return;
      }
      w = philox(TAG_PHANTOM, (uint64_t)ch, (uint64_t)j, att, seed, 0);
      x = 2.0 * unit53(w.v[0]) - 1.0;
      y = 2.0 * unit53(w.v[1]) - 1.0;
      s = x * x + y * y;
    }
    const double sq = sqrt(s);
    const double cph = x / sq, sph = y / sq;
    const double sth = sqrt(1.0 - cth * cth);
    const double sg = t2 >= 0.0 ? 1.0 : -1.0;
    const double aa = -1.0 / (sg + t2);
    const double bb = t0 * t1 * aa;
    const double e10 = 1.0 + sg * t0 * t0 * aa, e11 = sg * bb, e12 = -sg * t0;
    const double e20 = bb, e21 = sg + t1 * t1 * aa, e22 = -t1;
    const double n0 = cth * t0 + sth * (cph * e10 + sph * e20);
    const double n1 = cth * t1 + sth * (cph * e11 + sph * e21);
    const double n2 = cth * t2 + sth * (cph * e12 + sph * e22);
    const double q = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    t0 = n0 / q;
    t1 = n1 / q;
    t2 = n2 / q;
    p0 = p0 + bond * t0;
    p1 = p1 + bond * t1;
    p2 = p2 + bond * t2;
    rc[3 * j] = p0;
    rc[3 * j + 1] = p1;
    rc[3 * j + 2] = p2;
  }
}

// wrap caller positions into [0, L) and fold whole boxes into the image
// counters (the host-side rule, same FP64 operations); counts non-finite
// coordinates
__global__ void k_wrap(double *r, int32_t *img, int64_t n3, double L0, double L1, double L2,
                       unsigned long long *bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const int a = (int)(i % 3);
  const double L = a == 0 ? L0 : (a == 1 ? L1 : L2);
  double x = r[i];
  if (!isfinite(x)) {
    atomicAdd(bad, 1ull);
    return;
  }
  const double f = floor(x / L);
  x -= f * L;
  if (x >= L) x -= L;
  if (x < 0) x = 0;
  r[i] = x;
  img[i] += (int32_t)f;
}

// g1 table, one block: thread (k, j) adds the squared displacements of the
// middle beads over the lag j P^k (chains in order, (d0 d0 + d1 d1) + d2 d2)
// when sweep t is an origin multiple of P^k and the earlier snapshot exists;
// then every level whose period divides t stores the current snapshot in
// slot (t / P^k) mod P, which no lag of this sweep reads
__global__ void k_g1_track(const G1Track G) {
  const int64_t nch = G.n / G.N;
  const int nlag = G.K * (G.P - 1);
  for (int q = threadIdx.x; q < nlag; q += blockDim.x) {
    const int k = q / (G.P - 1), j = q % (G.P - 1) + 1;
    const int64_t pk = G.Pk[k];
    if (G.t % pk != 0 || G.t / pk < j) continue;
    const int64_t slot = (G.t / pk - j) % G.P;
    const double *old = G.ring + (k * (int64_t)G.P + slot) * nch * 3;
    double s = 0.0;
    for (int64_t ch = 0; ch < nch; ++ch) {
      const int64_t b = ch * G.N + G.N / 2;
      const double u0 = G.r[3 * b] + (double)G.img[3 * b] * G.L[0];
      const double u1 = G.r[3 * b + 1] + (double)G.img[3 * b + 1] * G.L[1];
      const double u2 = G.r[3 * b + 2] + (double)G.img[3 * b + 2] * G.L[2];
      const double d0 = u0 - old[3 * ch], d1 = u1 - old[3 * ch + 1], d2 = u2 - old[3 * ch + 2];
      s = s + ((d0 * d0 + d1 * d1) + d2 * d2);
    }
    G.sum[q] = G.sum[q] + s;
    G.cnt[q] += 1ull;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < (int64_t)G.K * nch; i += blockDim.x) {
    const int k = (int)(i / nch);
    const int64_t ch = i % nch;
    const int64_t pk = G.Pk[k];
    if (G.t % pk != 0) continue;
    const int64_t slot = (G.t / pk) % G.P;
    double *dst = G.ring + ((k * (int64_t)G.P + slot) * nch + ch) * 3;
    const int64_t b = ch * G.N + G.N / 2;
#pragma unroll
    for (int a = 0; a < 3; ++a) dst[a] = G.r[3 * b + a] + (double)G.img[3 * b + a] * G.L[a];
  }
}

__global__ void k_po_advance(const unsigned long long *count, int64_t *ctr) {
  if (*count) {
    ctr[0] += 1;
    ctr[1] += 1;
  }
}

}  // namespace

cudaError_t launch_po_advance(const unsigned long long *count, int64_t *ctr, cudaStream_t s) {
  k_po_advance<<<1, 1, 0, s>>>(count, ctr);
  return cudaGetLastError();
}

cudaError_t launch_g1_track(const G1Track &G, cudaStream_t s) {
  k_g1_track<<<1, 256, 0, s>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_wrap(double *r, int32_t *img, int64_t n, const double L[3],
                        unsigned long long *bad, cudaStream_t s) {
  const int64_t n3 = 3 * n;
  if (n3 > 0) k_wrap<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>(r, img, n3, L[0], L[1], L[2], bad);
  return cudaGetLastError();
}

cudaError_t launch_po_flags(const ObsParams &O, double thr, uint8_t *flag,
                            unsigned long long *count, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (O.n > 0) k_po_flags<<<(unsigned)((O.n + 255) / 256), 256, 0, s>>>(O, thr, flag, count);
  return cudaGetLastError();
}

cudaError_t launch_phantom(int64_t nch, int N, const double L[3], double bond, double ct,
                           uint64_t seed, double *r, unsigned long long *bad, cudaStream_t s) {
  if (nch > 0) k_phantom<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(nch, N, L[0], L[1], L[2], bond, ct, seed, r, bad);
  return cudaGetLastError();
}

cudaError_t launch_obs(const ObsParams &O, cudaStream_t s) {
  const int64_t nch = O.n / O.N;
  if (nch > 0) k_chains<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(O);
  if (O.n > 0 && O.cr) k_overlaps<<<(unsigned)((O.n + 127) / 128), 128, 0, s>>>(O);
  return cudaGetLastError();
}

cudaError_t launch_g1_snapshot(const ObsParams &O, double *g1ref, cudaStream_t s) {
  const int64_t nch = O.n / O.N;
  if (nch > 0) k_snapshot<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(O, g1ref);
  return cudaGetLastError();
}

cudaError_t launch_lattice(const int32_t dims[3], double a, double jitter, uint64_t seed,
                           uint64_t replica, double *r, int64_t n, cudaStream_t s) {
  if (n > 0)
    k_lattice<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dims[0], dims[1], dims[2], a, jitter,
                                                         seed, replica, r, n);
  return cudaGetLastError();
}

}  // namespace ecmc
