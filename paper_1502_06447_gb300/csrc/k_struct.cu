// Chain structure of the current state (arXiv:1502.06447, Sec. IV: radius
// of gyration and the relative MSD g2 of the middle bead; Appendix A: the
// moment of inertia tensor of a chain, its shape descriptors, and the
// end-to-end distance distribution W(R); Sec. II.B: mean-square internal
// distances R^2(n)).
//
// Positions along a chain come from minimum-image bonds: u_0 = 0,
// u_{j+1} = u_j + minimg(r_{j+1} - r_j).  The gyration tensor
// S = (1/N) sum_j (u_j - U)(u_j - U)^T with U = (1/N) sum_j u_j; the
// moment of inertia tensor is N (Tr S 1 - S), so its eigenvalue
// combinations follow from those of S.  Every sum runs in index order
// (beads, then chains), so all sums, S, R^2(n) and W(R) are reproducible
// bit for bit; the eigenvalues come from a cyclic Jacobi iteration.
#include <cuda_runtime.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

// Eigenvalues of a symmetric 3x3 matrix, ascending: cyclic Jacobi rotations
// (Rutishauser's formulation: t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (a_qq - a_pp) / (2 a_pq)), until the off-diagonal part is below
// 1e-18 of the diagonal or after 12 sweeps.
__device__ void sym3_eigen(double a00, double a01, double a02, double a11, double a12, double a22,
                           double &l0, double &l1, double &l2) {
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = fabs(a01) + fabs(a02) + fabs(a12);
    if (off <= 1e-18 * (fabs(a00) + fabs(a11) + fabs(a22)) || off == 0.0) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      // (p, q) = (0, 1), (0, 2), (1, 2); r is the third index
      double &app = pq == 2 ? a11 : a00;
      double &aqq = pq == 0 ? a11 : a22;
      double &apq = pq == 0 ? a01 : (pq == 1 ? a02 : a12);
      double &arp = pq == 0 ? a02 : (pq == 1 ? a01 : a01);  // a_rp
      double &arq = pq == 0 ? a12 : (pq == 1 ? a12 : a02);  // a_rq
      if (apq == 0.0) continue;
      const double theta = (aqq - app) / (2.0 * apq);
      double t;
      if (fabs(theta) > 1e150) {
        t = 0.5 / theta;
      } else {
        t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
        if (theta < 0.0) t = -t;
      }
      const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      app = app - t * apq;
      aqq = aqq + t * apq;
      apq = 0.0;
      const double xp = arp, xq = arq;
      arp = c * xp - s * xq;
      arq = s * xp + c * xq;
    }
  }
  // ascending order of the diagonal
  double x = a00, y = a11, z = a22, w;
  if (x > y) { w = x; x = y; y = w; }
  if (y > z) { w = y; y = z; z = w; }
  if (x > y) { w = x; x = y; y = w; }
  l0 = x;
  l1 = y;
  l2 = z;
}

// one thread per chain: positions along the chain (into u), the gyration
// tensor and its shape values, the middle bead relative to the centre of
// mass, g2's summand, |R_e|^2 and the end-to-end bin
__global__ void k_struct_chain(const StructParams S) {
  const int64_t ch = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nch = S.n / S.N;
  if (ch >= nch) return;
  const int N = S.N;
  const double *rc = S.r + 3 * ch * N;
  double *uc = S.u + 3 * ch * N;
  double u0 = 0.0, u1 = 0.0, u2 = 0.0;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;  // sums of u for the centre of mass
  uc[0] = uc[1] = uc[2] = 0.0;
  t0 = t0 + u0;
  t1 = t1 + u1;
  t2 = t2 + u2;
  for (int j = 0; j + 1 < N; ++j) {
    u0 = u0 + wrap_d(rc[3 * (j + 1)] - rc[3 * j], S.L[0], S.half[0]);
    u1 = u1 + wrap_d(rc[3 * (j + 1) + 1] - rc[3 * j + 1], S.L[1], S.half[1]);
    u2 = u2 + wrap_d(rc[3 * (j + 1) + 2] - rc[3 * j + 2], S.L[2], S.half[2]);
    uc[3 * (j + 1)] = u0;
    uc[3 * (j + 1) + 1] = u1;
    uc[3 * (j + 1) + 2] = u2;
    t0 = t0 + u0;
    t1 = t1 + u1;
    t2 = t2 + u2;
  }
  const double U0 = t0 / (double)N, U1 = t1 / (double)N, U2 = t2 / (double)N;
  double s00 = 0.0, s01 = 0.0, s02 = 0.0, s11 = 0.0, s12 = 0.0, s22 = 0.0;
  for (int j = 0; j < N; ++j) {
    const double d0 = uc[3 * j] - U0, d1 = uc[3 * j + 1] - U1, d2 = uc[3 * j + 2] - U2;
    s00 = s00 + d0 * d0;
    s01 = s01 + d0 * d1;
    s02 = s02 + d0 * d2;
    s11 = s11 + d1 * d1;
    s12 = s12 + d1 * d2;
    s22 = s22 + d2 * d2;
  }
  s00 = s00 / (double)N;
  s01 = s01 / (double)N;
  s02 = s02 / (double)N;
  s11 = s11 / (double)N;
  s12 = s12 / (double)N;
  s22 = s22 / (double)N;
  const double T = (s00 + s11) + s22;
  const double P = ((s00 * s11 - s01 * s01) + (s00 * s22 - s02 * s02)) + (s11 * s22 - s12 * s12);
  double l0, l1, l2;
  sym3_eigen(s00, s01, s02, s11, s12, s22, l0, l1, l2);
  const int h = N / 2;
  const double m0 = uc[3 * h] - U0, m1 = uc[3 * h + 1] - U1, m2 = uc[3 * h + 2] - U2;
  double g2 = 0.0;
  if (S.mref) {
    const double e0 = m0 - S.mref[3 * ch], e1 = m1 - S.mref[3 * ch + 1], e2 = m2 - S.mref[3 * ch + 2];
    g2 = (e0 * e0 + e1 * e1) + e2 * e2;
  }
  const double re2 = (u0 * u0 + u1 * u1) + u2 * u2;
  if (S.hist && S.nbins > 0) {
    int64_t b = (int64_t)floor(sqrt(re2) / S.dR);
    if (b >= S.nbins) b = S.nbins - 1;
    atomicAdd(&S.hist[b], 1ull);
  }
  double *o = S.rec + STRUCT_REC * ch;
  o[0] = T;
  o[1] = l0;
  o[2] = l1;
  o[3] = l2;
  o[4] = l2 - 0.5 * (l0 + l1);     // asphericity
  o[5] = l1 - l0;                  // acylindricity
  o[6] = 1.0 - 3.0 * P / (T * T);  // shape anisotropy
  o[7] = 4.0 * (T * T - 3.0 * P);  // 4 b^2 + 3 c^2
  o[8] = g2;
  o[9] = re2;
  o[10] = m0;
  o[11] = m1;
  o[12] = m2;
}

// R^2(n) partial sums: thread (chain, n) adds |u_{j+n} - u_j|^2 over j
__global__ void k_struct_r2n(const StructParams S) {
  const int N = S.N;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nch = S.n / N;
  if (t >= nch * (N - 1)) return;
  const int64_t ch = t / (N - 1);
  const int n = 1 + (int)(t % (N - 1));
  const double *uc = S.u + 3 * ch * N;
  double part = 0.0;
  for (int j = 0; j + n < N; ++j) {
    const double d0 = uc[3 * (j + n)] - uc[3 * j];
    const double d1 = uc[3 * (j + n) + 1] - uc[3 * j + 1];
    const double d2 = uc[3 * (j + n) + 2] - uc[3 * j + 2];
    part = part + ((d0 * d0 + d1 * d1) + d2 * d2);
  }
  S.part[ch * N + n] = part;
}

// sums over chains in chain order: the record columns (block 0) and R^2(n)
// (one thread per n)
__global__ void k_struct_sum(const StructParams S) {
  const int64_t nch = S.n / S.N;
  if (blockIdx.x == 0 && threadIdx.x < STRUCT_SUMS) {
    const int k = threadIdx.x;
    double s = 0.0;
    for (int64_t ch = 0; ch < nch; ++ch) s = s + S.rec[STRUCT_REC * ch + k];
    S.sums[k] = s;
  }
  if (!S.r2n) return;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= S.N) return;
  if (n == 0) {
    S.r2n[0] = 0.0;
    return;
  }
  double acc = 0.0;
  for (int64_t ch = 0; ch < nch; ++ch) acc = acc + S.part[ch * S.N + n];
  S.r2n[n] = acc / ((double)nch * (double)(S.N - n));
}

}  // namespace

cudaError_t launch_struct(const StructParams &S, cudaStream_t s) {
  const int64_t nch = S.n / S.N;
  if (nch <= 0 || S.N < 2) return cudaErrorInvalidValue;
  if (S.hist && S.nbins > 0) {
    cudaError_t e = cudaMemsetAsync(S.hist, 0, sizeof(unsigned long long) * (size_t)S.nbins, s);
    if (e != cudaSuccess) return e;
  }
  k_struct_chain<<<(unsigned)((nch + 127) / 128), 128, 0, s>>>(S);
  if (S.r2n) {
    const int64_t work = nch * (S.N - 1);
    k_struct_r2n<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(S);
  }
  const int nb = S.r2n ? (S.N + 127) / 128 : 1;
  k_struct_sum<<<nb, 128, 0, s>>>(S);
  return cudaGetLastError();
}

}  // namespace ecmc
