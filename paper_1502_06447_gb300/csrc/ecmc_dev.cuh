// Device/host primitives of the EC library: counter-based random numbers,
// the minimum image, the candidate kinds and the event digest.  The event
// geometry itself (arXiv:1502.06447, Sec. II, Eq. 1) lives in the kernels.
//
// Every FP64 expression is evaluated as written (the library is built with
// -fmad=false; fused multiply-adds only where written as __fma_rn), so the
// event sequence is a pure function of the input state and the Philox key.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define ECMC_HD __host__ __device__ __forceinline__
#else
#define ECMC_HD inline
#endif

namespace ecmc {

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64x64 -> 128-bit products of the even words with the round multipliers;
// the high halves are xor-ed into the odd words together with the key, the
// words rotate, and the key advances by the two Weyl increments.
struct u64x4 {
  uint64_t v[4];
};

ECMC_HD void mul128(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
#ifdef __CUDA_ARCH__
  hi = __umul64hi(a, b);
  lo = a * b;
#else
  unsigned __int128 p = (unsigned __int128)a * b;
  hi = (uint64_t)(p >> 64);
  lo = (uint64_t)p;
#endif
}

ECMC_HD u64x4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                     uint64_t k0, uint64_t k1) {
  const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
  const uint64_t w0 = 0x9E3779B97F4A7C15ull, w1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint64_t h0, l0, h1, l1;
    mul128(m0, c0, h0, l0);
    mul128(m1, c2, h1, l1);
    const uint64_t n0 = h1 ^ c1 ^ k0;
    const uint64_t n2 = h0 ^ c3 ^ k1;
    c0 = n0;
    c1 = l1;
    c2 = n2;
    c3 = l0;
    k0 += w0;
    k1 += w1;
  }
  u64x4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// random-number layout: key (seed, replica); counter (tag | ec << 8, sweep,
// unit, attempt).  Tags: 1 start bead + direction, 2 tile shift, 3 swap,
// 4 lattice jitter, 5 phantom chains, 6 spring energies (counter word 3 =
// the event index within the EC).
enum : uint64_t {
  TAG_START = 1, TAG_SHIFT = 2, TAG_SWAP = 3, TAG_JITTER = 4, TAG_PHANTOM = 5, TAG_SPRING = 6
};

// top 53 bits -> [0,1)
ECMC_HD double unit53(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

// floor(w * m / 2^64) in [0, m)
ECMC_HD int64_t scale_below(uint64_t w, uint64_t m) {
  uint64_t hi, lo;
  mul128(w, m, hi, lo);
  (void)lo;
  return (int64_t)hi;
}

// ---------------------------------------------------------------- geometry
// minimum image of one coordinate difference (|d| < L on input)
ECMC_HD double wrap_d(double d, double L, double half) {
  if (d > half) return d - L;
  if (d < -half) return d + L;
  return d;
}

// Candidate kinds in tie-break order: an exact tie in x goes to the smaller
// kind, then to the smaller partner id.
enum : int { KIND_END = 0, KIND_PASS = 1, KIND_WALL = 2, KIND_HS = 3, KIND_TETHER = 4 };

// ---------------------------------------------------------------- springs
// Bead-spring chains (Sec. II, ECs with pair potentials): the pieces the EC
// kernels need for a harmonic bond (k/2)(b - sigma)^2.  Host and device
// share them, so the host can check them against other implementations.
#ifdef __CUDA_ARCH__
#define EC_FMA(a, b, c) __fma_rn(a, b, c)
#else
#define EC_FMA(a, b, c) fma(a, b, c)
#endif

// Natural logarithm of u in (0, 1]: u = m 2^e with m in [sqrt(1/2), sqrt(2)),
// log u = e ln 2 + 2 atanh(z), z = (m - 1)/(m + 1), atanh(z)/z =
// sum_{n=0..14} z^(2n)/(2n + 1) by Horner's rule, ln 2 rounded to double.
// Only +, -, *, / and exact bit moves: every implementation taking these
// steps gets the same bits (within a few ulp of the exact logarithm).
ECMC_HD double ec_log(double u) {
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

// Boltzmann energy of one bond at one event from a Philox word:
// dE = -log(u), u = 1 - unit53(w) in (0, 1]
ECMC_HD double spring_dE(uint64_t w) { return -ec_log(1.0 - unit53(w)); }

// Spring event: a pivot at separation d = r_pivot - r_bonded moving along
// unit v may go on until the energy its move adds reaches dE.  Hard spheres
// keep b >= sigma, so the energy falls up to the closest approach along the
// path and rises after it (or from the start when d.v >= 0); dE is spent
// on the rise: b_t = sigma + sqrt((b_s - sigma)^2 + 2 dE / k) with b_s the
// bond length where the rise starts, x = -d.v + sqrt(b_t^2 - |d_perp|^2).
ECMC_HD double spring_x(double d0, double d1, double d2, double v0, double v1, double v2,
                        double sigma, double k, double dE, double &dv) {
  dv = EC_FMA(d2, v2, EC_FMA(d1, v1, d0 * v0));
  const double dd = EC_FMA(d2, d2, EC_FMA(d1, d1, d0 * d0));
  double perp2 = EC_FMA(-dv, dv, dd);
  if (perp2 < 0.0) perp2 = 0.0;
  const double bs = dv < 0.0 ? sqrt(perp2) : sqrt(dd);
  const double e = bs - sigma;
  const double bt = sigma + sqrt(e * e + 2.0 * dE / k);
  // b_t >= b_s >= |d_perp| exactly; rounding can leave the radicand a few
  // ulp below zero when dE ~ 0 and the path grazes the closest approach
  double rad = bt * bt - perp2;
  if (rad < 0.0) rad = 0.0;
  double x = -dv + sqrt(rad);
  if (x < 0.0) x = 0.0;
  return x;
}

ECMC_HD void fnv_mix(uint64_t &h, uint64_t w) {
  h ^= w;
  h *= 0x100000001B3ull;
}

#ifdef __CUDACC__
// FP32 bounds on a square root and a quotient from the hardware's fast
// approximations.  rsqrtf errs by at most 2 ulp and __fdividef (divisor in
// [2^-126, 2^126]) by at most 2 ulp (CUDA's accuracy tables), so after the
// final product the relative error is below 4e-7 and the factors 1 -+ 1e-6
// give a lower and an upper bound.  sqrt arguments are raised to 1e-30
// inside rsqrtf: this keeps 0 finite and moves a result by less than 1e-15
// in absolute terms, far inside the screen's margin eps_v.
__device__ __forceinline__ float sqrt_lo(float y) { return y * rsqrtf(fmaxf(y, 1e-30f)) * 0.999999f; }
__device__ __forceinline__ float sqrt_hi(float y) { return y * rsqrtf(fmaxf(y, 1e-30f)) * 1.000001f; }
__device__ __forceinline__ float div_lo(float a, float b) { return __fdividef(a, b) * 0.999999f; }
__device__ __forceinline__ float div_hi(float a, float b) { return __fdividef(a, b) * 1.000001f; }

#endif

}  // namespace ecmc
