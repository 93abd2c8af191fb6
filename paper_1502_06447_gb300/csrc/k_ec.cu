// Event-chain kernels (arXiv:1502.06447, Sec. II: EC move, with hard tethers
// or harmonic bead springs; Sec. II.A: tile-joint decomposition with
// reflections; Sec. II.C: swap move).
//
// One group of G lanes (G = 32, 16, 8 or 4) runs the ECs of one tile; the
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
// arithmetic of the plain definition.  In the domain mode the hard-sphere
// slots [0, m + j1) also sit in a local cell grid of side >= one free
// flight's reach (s_cap + 1.01 sigma), kept current as beads move, and an
// event scans only the 27 cells around the pivot; the serial mode scans all
// beads.
//
// GB300's FP64 pipe is the scarce resource, so FP64 comparisons are done on
// the bit patterns with integer instructions (same results), and in the
// screened form (F32) every candidate — contact, tether, wall — is first
// bounded in FP32 from tile-local shadows; only those whose lower bound can
// reach the smallest upper bound U are evaluated in FP64, in rounds shared by
// all lanes.  A candidate left out cannot be the winner: the winner's exact x
// is <= U and every lower bound is <= its candidate's exact x.
#include "ec_device.cuh"

namespace ecmc {
namespace {

template <int G, bool F32, bool BATCH>
__global__ void __launch_bounds__(128) ec_kernel(const ECParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  // push-off run from the device: nothing to do once no bead overlaps
  if (P.po_count && *P.po_count == 0ull) return;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int gbase = lane & ~(G - 1);
  const int gib = threadIdx.x / G;
  const int gpb = blockDim.x / G;
  const int gunit = blockIdx.x * gpb + gib;  // unit over all replicas
  // the replica of this unit (batch) and the unit's tile within it
  const RepParams *rp = nullptr;
  int unit = gunit;
  if (BATCH) {
    int lo = 0, hi = P.n_reps - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (P.reps[mid].unit_off <= gunit) lo = mid;
      else hi = mid - 1;
    }
    rp = P.reps + lo;
    unit = gunit - (int)rp->unit_off;
  }
#define SYS(f) (BATCH ? rp->f : P.f)
  double *const Rr = BATCH ? P.r + 3 * rp->bead_off : P.r;
  int32_t *const Ri = BATCH ? P.img + 3 * rp->bead_off : P.img;
  const int32_t *const Rstart = BATCH ? P.cstart + rp->cell_off : P.cstart;
  const uint64_t Rkey = BATCH ? rp->replica : P.replica;
  const int64_t sweep = P.sweep_dev ? *P.sweep_dev : P.sweep;
  const int S = P.stage_cap;
  const int NC = P.domain ? (BATCH ? P.ncl_max : SYS(lg)[0] * SYS(lg)[1] * SYS(lg)[2]) : 0;
  const int M = (F32 && P.domain) ? P.m_cap : S;
  Stage st = carve(smem + (size_t)gib * group_bytes(S, M, M, NC), S, M, M, NC);
#ifdef ECMC_CHECKED
  st.status = P.status;
  st.nglob = BATCH ? rp->n_beads : P.n;
#endif
  bool live = gunit < P.n_units;
  const uint64_t hb0 = dbits(SYS(half)[0]), hb1 = dbits(SYS(half)[1]), hb2 = dbits(SYS(half)[2]);
  LGrid LG;
  LG.g0 = SYS(lg)[0];
  LG.g1 = SYS(lg)[1];
  LG.g2 = SYS(lg)[2];
  LG.org = SYS(lorg);
  LG.inv0 = SYS(linv)[0];
  LG.inv1 = SYS(linv)[1];
  LG.inv2 = SYS(linv)[2];

  // tile geometry (domain) or the whole box (serial); corner = shift + k T
  int tk[3] = {0, 0, 0};
  double c0 = 0.0, c1 = 0.0, c2 = 0.0;
  if (P.domain && live) {
    tk[0] = unit % SYS(D)[0];
    tk[1] = (unit / SYS(D)[0]) % SYS(D)[1];
    tk[2] = unit / (SYS(D)[0] * SYS(D)[1]);
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)sweep, 0, 0, P.seed, Rkey);
    c0 = unit53(w.v[0]) * SYS(T)[0] + (double)tk[0] * SYS(T)[0];
    c1 = unit53(w.v[1]) * SYS(T)[1] + (double)tk[1] * SYS(T)[1];
    c2 = unit53(w.v[2]) * SYS(T)[2] + (double)tk[2] * SYS(T)[2];
  }

  // ------------------------------------------------------------ staging
  int m = 0, j1 = 0, ns = 0;
  stage_tile<G, F32, BATCH>(P, rp, st, gl, live, unit, c0, c1, c2, Rr, Rstart, S, M, M, NC, LG, m,
                            j1, ns);
  const int nhs = m + j1;
  const int nhs_max = __reduce_max_sync(FULL, nhs);

  // ------------------------------------------------------------ ECs
  // A tile whose halo lies inside (0, L) on an axis never needs the minimum
  // image or a wrap on that axis: every position it touches stays in one
  // periodic image.  Those axes skip the wrap code entirely.
  bool wr0 = true, wr1 = true, wr2 = true;
  if (P.domain) {
    wr0 = !(c0 - P.halo_te > 0.0 && c0 + SYS(W)[0] + P.halo_te < SYS(L)[0]);
    wr1 = !(c1 - P.halo_te > 0.0 && c1 + SYS(W)[1] + P.halo_te < SYS(L)[1]);
    wr2 = !(c2 - P.halo_te > 0.0 && c2 + SYS(W)[2] + P.halo_te < SYS(L)[2]);
  }
  const float cf0 = (float)c0, cf1 = (float)c1, cf2 = (float)c2;
  const float Lh0 = 0.5f * (float)SYS(L)[0], Lh1 = 0.5f * (float)SYS(L)[1], Lh2 = 0.5f * (float)SYS(L)[2];
  const int n_ec = P.ecs_per_tile;
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
  const float Lf0 = (float)SYS(L)[0], Lf1 = (float)SYS(L)[1], Lf2 = (float)SYS(L)[2];
  const float Wf0 = (float)SYS(W)[0], Wf1 = (float)SYS(W)[1], Wf2 = (float)SYS(W)[2];
  const float INF = __int_as_float(0x7f800000);
  const double DINF = __longlong_as_double(0x7ff0000000000000ll);
  double lift_all = 0.0, refl_all = 0.0, disp_all = 0.0;
  unsigned long long cnt[ECMC_NEV];
#pragma unroll
  for (int k = 0; k < ECMC_NEV; ++k) cnt[k] = 0;
  unsigned long long tried = 0, confirmed = 0, nev_all = 0, ecs_done = 0;
  constexpr int ITEMS = G >= 8 ? 1 : 2;  // special candidates per lane

  // push-off: one EC from every flagged motile bead of the tile, in id order
  int n_ec_g = n_ec;
  if (P.po_flag) {
    int f = 0;
    for (int s = gl; s < m; s += G) f += P.po_flag[st.id[s]] ? 1 : 0;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) f += __shfl_xor_sync(FULL, f, off);
    n_ec_g = live ? f : 0;
  }
  const int n_ec_run = P.po_flag ? __reduce_max_sync(FULL, n_ec_g) : n_ec;
  for (int e = 0; e < n_ec_run; ++e) {
    bool active = live && m > 0 && e < n_ec_g;
    const uint64_t r0 = P.domain ? (TAG_START | ((uint64_t)e << 8)) : TAG_START;
    const uint64_t r1 = P.domain ? (uint64_t)sweep : 0;
    const uint64_t r2 = P.domain ? (uint64_t)unit : (uint64_t)(sweep + e);
    int p = 0;
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (active) {
      u64x4 w = philox(r0, r1, r2, 0, P.seed, Rkey);
      p = (int)scale_below(w.v[0], (uint64_t)m);
      if (P.po_flag) {
        // the e-th flagged motile slot (slots are in id order)
        for (int s = 0, f = 0; s < m; ++s) {
          if (!P.po_flag[st.id[s]]) continue;
          if (f == e) {
            p = s;
            break;
          }
          ++f;
        }
      }
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
          w = philox(r0, r1, r2, att, P.seed, Rkey);
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
    double lift = 0.0;

    while (__any_sync(FULL, active)) {
      if (active && nev >= P.event_cap) {
        if (gl == 0) set_status(P.status, DEV_STUCK);
        active = false;
      }
      double bx = DINF;  // lane-local best exactly evaluated candidate
      uint64_t bkey = ~0ull;
      double bdv = 0.0;
      const unsigned nbw = active ? st.nb[p] : 0xFFFFFFFFu;
      int pc0 = 0, pc1 = 0, pc2 = 0;
      if (P.domain) lcell(LG, pf0, pf1, pf2, pc0, pc1, pc2);
      const int n_ovf = P.domain ? st.hdr[4] : 0;
      // --------- special candidates: item 0 end/pass, 1-2 tethers, 3-5 walls
      float ubl = INF;
      int spk[ITEMS], sps[ITEMS];
      float spl[ITEMS];
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        spk[r] = -1;
        sps[r] = -1;
        spl[r] = INF;
        const int it = gl + r * G;
        if (!active || it >= 6) continue;
        if (it == 0) {
          if (dbits(P.s_cap) < dbits(xrem)) {
            bx = P.s_cap;
            bkey = make_key(KIND_PASS, 0, 0);
          } else {
            bx = xrem;
            bkey = make_key(KIND_END, 0, 0);
          }
          if (F32) ubl = fminf(ubl, __double2float_ru(bx));
        } else if (it <= 2) {
          const int t = it == 1 ? nb_prev(nbw) : nb_next(nbw);
          if (t < 0) continue;
          if (P.k_spring > 0.0) {
            // bead spring (Sec. II, ECs with pair potentials): a fresh
            // Boltzmann energy per bond and event, spent on the rising part
            // of the path; always evaluated in FP64, and in the screened
            // form its exact x bounds U from above
            const u64x4 w = philox(TAG_SPRING | ((uint64_t)(P.domain ? e : 0) << 8), r1, r2,
                                   (uint64_t)nev, P.seed, Rkey);
            double kx, ky, kz, dv;
            pos64(st, Rr, t, !F32 || t < m, kx, ky, kz);
            // (a spring partner may lie beyond the tile's halo, across the
            // periodic boundary: always the minimum image)
            const double x = spring_x(wrap_i(q0 - kx, SYS(L)[0], hb0), wrap_i(q1 - ky, SYS(L)[1], hb1),
                                      wrap_i(q2 - kz, SYS(L)[2], hb2), v0, v1, v2, P.sigma,
                                      P.k_spring, spring_dE(it == 1 ? w.v[0] : w.v[1]), dv);
            const uint64_t key = make_key(KIND_TETHER, st.id[t], t);
            if (better(x, key, bx, bkey)) {
              bx = x;
              bkey = key;
              bdv = dv;
            }
            if (F32) ubl = fminf(ubl, __double2float_ru(x));
            continue;
          }
          if (!F32) {
            double dv;
            const double x = quad_x(true, wrapc(q0 - st.px[t], SYS(L)[0], hb0, wr0),
                                    wrapc(q1 - st.py[t], SYS(L)[1], hb1, wr1),
                                    wrapc(q2 - st.pz[t], SYS(L)[2], hb2, wr2), v0, v1, v2, P.b2, dv);
            const uint64_t key = make_key(KIND_TETHER, st.id[t], t);
            if (better(x, key, bx, bkey)) {
              bx = x;
              bkey = key;
              bdv = dv;
            }
          } else {
            float d0 = pf0 - st.fx[t], d1 = pf1 - st.fy[t], d2 = pf2 - st.fz[t];
            if (!P.domain) {
              d0 = wrapf(d0, Lf0);
              d1 = wrapf(d1, Lf1);
              d2 = wrapf(d2, Lf2);
            }
            const float dd = __fmaf_rn(d2, d2, __fmaf_rn(d1, d1, d0 * d0));
            const float dv = __fmaf_rn(d2, vf2, __fmaf_rn(d1, vf1, d0 * vf0));
            const float rad = b2f - (dd - dv * dv);
            const float lo = -dv - eps_v + sqrt_lo(fmaxf(rad - eps_d, 0.f));
            const float hi = -dv + eps_v + sqrt_hi(fmaxf(rad + eps_d, 0.f));
            spl[r] = fmaxf(lo, 0.f);
            ubl = fminf(ubl, fmaxf(hi, 0.f) + 1e-6f);
            spk[r] = KIND_TETHER;
            sps[r] = t;
          }
        } else if (P.domain) {
          const int a = it - 3;
          const double va = a == 0 ? v0 : (a == 1 ? v1 : v2);
          if (!nonzero(va)) continue;
          if (!F32) {
            const double qa = a == 0 ? q0 : (a == 1 ? q1 : q2);
            const double ca = a == 0 ? c0 : (a == 1 ? c1 : c2);
            const double loc = wrapc(qa - ca, SYS(L)[a], a == 0 ? hb0 : (a == 1 ? hb1 : hb2),
                                     a == 0 ? wr0 : (a == 1 ? wr1 : wr2));
            double x = posv(va) ? (SYS(W)[a] - loc) / va : (0.0 - loc) / va;
            if (neg(x)) x = 0.0;
            const uint64_t key = make_key(KIND_WALL, a, 0);
            if (better(x, key, bx, bkey)) {
              bx = x;
              bkey = key;
            }
          } else {
            const float vfa = a == 0 ? vf0 : (a == 1 ? vf1 : vf2);
            const float pfa = a == 0 ? pf0 : (a == 1 ? pf1 : pf2);
            const float Wfa = a == 0 ? Wf0 : (a == 1 ? Wf1 : Wf2);
            const float dist = posv(va) ? Wfa - pfa : pfa;
            const float av = fabsf(vfa);
            if (av >= 1e-30f) {
              spl[r] = div_lo(fmaxf(dist - eps_v, 0.f), av);
              ubl = fminf(ubl, div_hi(fmaxf(dist, 0.f) + eps_v, av));
            } else {
              spl[r] = 0.f;  // |v_a| below FP32 range: confirm in FP64
            }
            spk[r] = KIND_WALL;
            sps[r] = a;
          }
        }
      }
      // --------- hard-sphere obstacles
      int ks0 = -1, ks1 = -1;
      float kl0 = INF, kl1 = INF;
      bool kovf = false;
      if (P.domain) {
        // the 27 cells around the pivot (item 27: the overflow list)
        for (int ci = gl; ci < 28; ci += G) {
          if (!active) break;
          int n;
          const unsigned short *lst;
          if (ci == 27) {
            n = n_ovf;
            lst = st.ovf;
          } else {
            const int x = pc0 + ci % 3 - 1, y = pc1 + (ci / 3) % 3 - 1, z = pc2 + ci / 9 - 1;
            if (x < 0 || y < 0 || z < 0 || x >= LG.g0 || y >= LG.g1 || z >= LG.g2) continue;
            const unsigned short *c = st.cell + 8 * ((z * LG.g1 + y) * LG.g0 + x);
            if (F32) {
              screen_cell(Z, st, c, p, pf0, pf1, pf2, vf0, vf1, vf2, ubl, ks0, kl0, ks1, kl1, kovf);
              continue;
            }
            n = cell_n(c);
            lst = c + 2;
          }
          for (int i = 0; i < n; ++i) {
            const int k = lst[i];
            if (k == p) continue;
            if (!F32) {
              double dv;
              const double x = quad_x(false, wrapc(q0 - st.px[k], SYS(L)[0], hb0, wr0),
                                      wrapc(q1 - st.py[k], SYS(L)[1], hb1, wr1),
                                      wrapc(q2 - st.pz[k], SYS(L)[2], hb2, wr2), v0, v1, v2, P.sig2, dv,
                                      P.po_flag != nullptr);
              if (!neg(x)) {
                const uint64_t key = make_key(KIND_HS, st.id[k], k);
                if (better(x, key, bx, bkey)) {
                  bx = x;
                  bkey = key;
                  bdv = dv;
                }
              }
            } else {
              screen_hs(Z, pf0 - st.fx[k], pf1 - st.fy[k], pf2 - st.fz[k], vf0, vf1, vf2, k, ubl,
                        ks0, kl0, ks1, kl1, kovf);
            }
          }
        }
      } else {
        for (int k0 = 0; k0 < nhs_max; k0 += G) {
          const int k = k0 + gl;
          if (!(active && k < nhs && k != p)) continue;
          if (!F32) {
            double dv;
            const double x = quad_x(false, wrapc(q0 - st.px[k], SYS(L)[0], hb0, wr0),
                                    wrapc(q1 - st.py[k], SYS(L)[1], hb1, wr1),
                                    wrapc(q2 - st.pz[k], SYS(L)[2], hb2, wr2), v0, v1, v2, P.sig2, dv);
            if (!neg(x)) {
              const uint64_t key = make_key(KIND_HS, st.id[k], k);
              if (better(x, key, bx, bkey)) {
                bx = x;
                bkey = key;
                bdv = dv;
              }
            }
          } else {
            screen_hs(Z, wrapf(pf0 - st.fx[k], Lf0), wrapf(pf1 - st.fy[k], Lf1),
                      wrapf(pf2 - st.fz[k], Lf2), vf0, vf1, vf2, k, ubl, ks0, kl0, ks1, kl1, kovf);
          }
        }
      }
      if (F32) {
        const float U = group_minf<G>(ubl);
        // survivors of this lane, confirmed in FP64 in shared rounds
        int jq0 = -1, jq1 = -1, jq2 = -1, jq3 = -1;
        int nj = 0;
        auto push = [&](int v) {
          if (nj == 0) jq0 = v;
          else if (nj == 1) jq1 = v;
          else if (nj == 2) jq2 = v;
          else jq3 = v;
          ++nj;
        };
#pragma unroll
        for (int r = 0; r < ITEMS; ++r)
          if (spk[r] == KIND_TETHER && spl[r] <= U) push(sps[r] | (1 << 30));
        if (ks0 >= 0 && kl0 <= U) push(ks0);
        if (ks1 >= 0 && kl1 <= U) push(ks1);
        const int rounds = __reduce_max_sync(FULL, nj);
        for (int rr = 0; rr < rounds; ++rr) {
          if (rr < nj) {
            const int jb = rr == 0 ? jq0 : (rr == 1 ? jq1 : (rr == 2 ? jq2 : jq3));
            const bool te = (jb >> 30) & 1;
            const int k = jb & 0x3FFFFFFF;
            double kx, ky, kz, dv;
            pos64(st, Rr, k, !F32 || k < m, kx, ky, kz);
            const double x = quad_x(te, wrapc(q0 - kx, SYS(L)[0], hb0, wr0), wrapc(q1 - ky, SYS(L)[1], hb1, wr1),
                                    wrapc(q2 - kz, SYS(L)[2], hb2, wr2), v0, v1, v2,
                                    te ? P.b2 : P.sig2, dv);
            ++confirmed;
            if (!neg(x)) {
              const uint64_t key = make_key(te ? KIND_TETHER : KIND_HS, st.id[k], k);
              if (better(x, key, bx, bkey)) {
                bx = x;
                bkey = key;
                bdv = dv;
              }
            }
          }
        }
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
          if (!(spk[r] == KIND_WALL && spl[r] <= U)) continue;
          const int a = sps[r];
          const double va = a == 0 ? v0 : (a == 1 ? v1 : v2);
          const double qa = a == 0 ? q0 : (a == 1 ? q1 : q2);
          const double ca = a == 0 ? c0 : (a == 1 ? c1 : c2);
          const double loc = wrapc(qa - ca, SYS(L)[a], a == 0 ? hb0 : (a == 1 ? hb1 : hb2),
                                     a == 0 ? wr0 : (a == 1 ? wr1 : wr2));
          double x = posv(va) ? (SYS(W)[a] - loc) / va : (0.0 - loc) / va;
          if (neg(x)) x = 0.0;
          ++confirmed;
          const uint64_t key = make_key(KIND_WALL, a, 0);
          if (better(x, key, bx, bkey)) {
            bx = x;
            bkey = key;
          }
        }
        if (kovf) {
          // more than two possible winners in this lane: evaluate again
          auto rescan = [&](int k) {
            if (k == p || k == ks0 || k == ks1) return;
            bool possible;
            float d0 = pf0 - st.fx[k], d1 = pf1 - st.fy[k], d2 = pf2 - st.fz[k];
            if (!P.domain) {
              d0 = wrapf(d0, Lf0);
              d1 = wrapf(d1, Lf1);
              d2 = wrapf(d2, Lf2);
            }
            const float lb = screen_lb(Z, d0, d1, d2, vf0, vf1, vf2, possible);
            if (!possible || lb > U) return;
            double kx, ky, kz, dvx;
            pos64(st, Rr, k, !F32 || k < m, kx, ky, kz);
            const double x = quad_x(false, wrapc(q0 - kx, SYS(L)[0], hb0, wr0),
                                    wrapc(q1 - ky, SYS(L)[1], hb1, wr1), wrapc(q2 - kz, SYS(L)[2], hb2, wr2),
                                    v0, v1, v2, P.sig2, dvx);
            ++confirmed;
            if (!neg(x)) {
              const uint64_t key = make_key(KIND_HS, st.id[k], k);
              if (better(x, key, bx, bkey)) {
                bx = x;
                bkey = key;
                bdv = dvx;
              }
            }
          };
          if (P.domain) {
            for (int ci = gl; ci < 28; ci += G) {
              int n;
              const unsigned short *lst;
              if (ci == 27) {
                n = n_ovf;
                lst = st.ovf;
              } else {
                const int x = pc0 + ci % 3 - 1, y = pc1 + (ci / 3) % 3 - 1, z = pc2 + ci / 9 - 1;
                if (x < 0 || y < 0 || z < 0 || x >= LG.g0 || y >= LG.g1 || z >= LG.g2) continue;
                const unsigned short *c = st.cell + 8 * ((z * LG.g1 + y) * LG.g0 + x);
                n = cell_n(c);
                lst = c + 2;
              }
              for (int i = 0; i < n; ++i) rescan(lst[i]);
            }
          } else {
            for (int k = gl; k < nhs; k += G) rescan(k);
          }
        }
      }
      // ---------------- winner of the group and its pre-flight d.v
      const uint64_t my_key = bkey;
      const uint64_t my_x = dbits(bx);
      group_argmin<G>(bx, bkey);
      const unsigned own = __ballot_sync(FULL, my_key == bkey && my_x == dbits(bx));
      const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1) << gbase);
      const int src = __ffs(own & gmask) - 1;
      const double wdv = __shfl_sync(FULL, bdv, src < 0 ? lane : src);
      __syncwarp();

      int np = p;
      if (active) {
        const double x = bx;
        const int kind = key_kind(bkey);
        const int slot = key_slot(bkey);
        const int64_t partner = (kind == KIND_END || kind == KIND_PASS) ? -1 : key_id(bkey);
        int di0 = 0, di1 = 0, di2 = 0;
        if (wr0) di0 = step_i(q0, x, v0, SYS(L)[0]);
        else q0 = __fma_rn(x, v0, q0);
        if (wr1) di1 = step_i(q1, x, v1, SYS(L)[1]);
        else q1 = __fma_rn(x, v1, q1);
        if (wr2) di2 = step_i(q2, x, v2, SYS(L)[2]);
        else q2 = __fma_rn(x, v2, q2);
        if (gl == 0 && (di0 | di1 | di2)) {
          if (di0) Ri[3 * (int64_t)pid] += di0;
          if (di1) Ri[3 * (int64_t)pid + 1] += di1;
          if (di2) Ri[3 * (int64_t)pid + 2] += di2;
        }
        ++nev;
        int out;
        bool swapped = false;
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
          // (r_target - r_pivot).v at contact = -(d.v) - x
          const double proj = -wdv - x;
          const bool motile = slot < m;
          if (!motile) {
            out = kind == KIND_HS ? ECMC_EV_HS_REFLECT : ECMC_EV_TE_REFLECT;
            refl_all = refl_all + proj;
            double kx, ky, kz;
            pos64(st, Rr, slot, !F32 || slot < m, kx, ky, kz);
            const bool sp = P.k_spring > 0.0 && kind == KIND_TETHER;
            mirror2(v0, v1, v2, wrapc(q0 - kx, SYS(L)[0], hb0, wr0 || sp),
                    wrapc(q1 - ky, SYS(L)[1], hb1, wr1 || sp), wrapc(q2 - kz, SYS(L)[2], hb2, wr2 || sp));
          } else if (kind == KIND_HS) {
            lift = lift + proj;
            if (P.swap_mode) {
              bool go;
              if (P.swap_mode == 1) {
                go = true;
              } else {
                if ((ncontact & 3) == 0)
                  swr = philox(TAG_SWAP | ((uint64_t)(P.domain ? e : 0) << 8), r1, r2,
                               (uint64_t)(ncontact >> 2), P.seed, Rkey);
                go = (swr.v[ncontact & 3] >> 11) < P.swap_thr;
              }
              ++ncontact;
              if (go) {
                ++tried;
                const double k0 = st.px[slot], k1 = st.py[slot], k2 = st.pz[slot];
                // every bond of both beads, positions exchanged, within b_max
                bool ok = true;
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                  const int a = side == 0 ? p : slot;
                  const double a0 = side == 0 ? k0 : q0;
                  const double a1 = side == 0 ? k1 : q1;
                  const double a2 = side == 0 ? k2 : q2;
                  const unsigned nbv = st.nb[a];
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
                      pos64(st, Rr, b, !F32 || b < m, b0, b1, b2);
                    }
                    const double e0 = wrapc(a0 - b0, SYS(L)[0], hb0, wr0);
                    const double e1 = wrapc(a1 - b1, SYS(L)[1], hb1, wr1);
                    const double e2 = wrapc(a2 - b2, SYS(L)[2], hb2, wr2);
                    const double dd = __fma_rn(e2, e2, __fma_rn(e1, e1, e0 * e0));
                    ok = ok && !(dbits(dd) > dbits(P.b2));
                  }
                }
                if (ok) {
                  swapped = true;
                  if (gl == 0) {
                    st.px[slot] = q0;
                    st.py[slot] = q1;
                    st.pz[slot] = q2;
                    const int kid = st.id[slot];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                      const int ti = Ri[3 * (int64_t)pid + a];
                      Ri[3 * (int64_t)pid + a] = Ri[3 * (int64_t)kid + a];
                      Ri[3 * (int64_t)kid + a] = ti;
                    }
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
#pragma unroll
        for (int k = 0; k < ECMC_NEV; ++k) cnt[k] += (out == k);
        // FP32 shadow of the moved pivot: FP32 position minus FP32 corner
        // (within the margins of the screen)
        float nf0, nf1, nf2;
        if (P.domain) {
          nf0 = (float)q0 - cf0;
          nf1 = (float)q1 - cf1;
          nf2 = (float)q2 - cf2;
          if (wr0) nf0 = nf0 > Lh0 ? nf0 - (float)SYS(L)[0] : (nf0 < -Lh0 ? nf0 + (float)SYS(L)[0] : nf0);
          if (wr1) nf1 = nf1 > Lh1 ? nf1 - (float)SYS(L)[1] : (nf1 < -Lh1 ? nf1 + (float)SYS(L)[1] : nf1);
          if (wr2) nf2 = nf2 > Lh2 ? nf2 - (float)SYS(L)[2] : (nf2 < -Lh2 ? nf2 + (float)SYS(L)[2] : nf2);
        } else {
          nf0 = (float)q0;
          nf1 = (float)q1;
          nf2 = (float)q2;
        }
        if (gl == 0) {
          fnv_mix(h, (uint64_t)pid);
          fnv_mix(h, ((uint64_t)(uint32_t)out << 32) | (uint64_t)(uint32_t)partner);
          fnv_mix(h, dbits(x));
          if (P.log) {
            const unsigned long long at = atomicAdd(P.log_n, 1ull);
            if ((int64_t)at < P.log_cap) {
              ecmc_event ev;
              ev.unit = P.rec_offset + (P.sweep_dev ? (sweep - P.rec_sweep0) * P.n_units * n_ec : 0) + (P.domain ? (int64_t)gunit * n_ec + e : (int64_t)e);
              ev.seq = (int32_t)(nev - 1);
              ev.pivot = pid;
              ev.kind = out;
              ev.pad = 0;
              ev.partner = partner;
              ev.x = x;
              P.log[at] = ev;
            }
          }
          st.px[p] = q0;
          st.py[p] = q1;
          st.pz[p] = q2;
          if (P.domain) {
            // keep the local grid current
            int a0, a1, a2, b0, b1, b2;
            const int oc = lcell(LG, pf0, pf1, pf2, a0, a1, a2);
            const int ncl = lcell(LG, nf0, nf1, nf2, b0, b1, b2);
            if (swapped) {
              const double o0 = st.px[slot], o1 = st.py[slot], o2 = st.pz[slot];
              float g0 = (float)o0 - cf0, g1 = (float)o1 - cf1, g2 = (float)o2 - cf2;
              if (wr0) g0 = g0 > Lh0 ? g0 - (float)SYS(L)[0] : (g0 < -Lh0 ? g0 + (float)SYS(L)[0] : g0);
              if (wr1) g1 = g1 > Lh1 ? g1 - (float)SYS(L)[1] : (g1 < -Lh1 ? g1 + (float)SYS(L)[1] : g1);
              if (wr2) g2 = g2 > Lh2 ? g2 - (float)SYS(L)[2] : (g2 < -Lh2 ? g2 + (float)SYS(L)[2] : g2);
              const int koc = lcell(LG, st.fx[slot], st.fy[slot], st.fz[slot], a0, a1, a2);
              const int knc = lcell(LG, g0, g1, g2, b0, b1, b2);
              lcell_remove(st, oc, p);
              lcell_remove(st, koc, slot);
              st.fx[slot] = g0;
              st.fy[slot] = g1;
              st.fz[slot] = g2;
              bool ok = lcell_insert(st, ncl, p);
              ok = lcell_insert(st, knc, slot) && ok;
              if (!ok) set_status(P.status, DEV_CAPACITY);
            } else if (oc != ncl) {
              lcell_remove(st, oc, p);
              if (!lcell_insert(st, ncl, p)) set_status(P.status, DEV_CAPACITY);
            }
          } else if (F32 && swapped) {
            st.fx[slot] = (float)st.px[slot];
            st.fy[slot] = (float)st.py[slot];
            st.fz[slot] = (float)st.pz[slot];
          }
          st.fx[p] = nf0;
          st.fy[p] = nf1;
          st.fz[p] = nf2;
        }
        pf0 = nf0;
        pf1 = nf1;
        pf2 = nf2;
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
        pf0 = st.fx[p];
        pf1 = st.fy[p];
        pf2 = st.fz[p];
      }
      __syncwarp();
    }
    // EC records
    if (live && m > 0) {
      lift_all = lift_all + lift;
      disp_all = disp_all + P.ell;  // the free flights of an EC add up to ell
      nev_all += (unsigned long long)nev;
      ++ecs_done;
      if (gl == 0 && P.rec_digest) {
        const int64_t idx = P.rec_offset + (P.sweep_dev ? (sweep - P.rec_sweep0) * P.n_units * n_ec : 0) + (P.domain ? (int64_t)gunit * n_ec + e : (int64_t)e);
        if (idx < P.rec_cap) {
          P.rec_digest[idx] = h;
          P.rec_lift[idx] = lift;
          P.rec_events[idx] = nev;
        }
      }
    }
  }
  // counters of this group's ECs
  if (F32) {
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) confirmed += __shfl_xor_sync(FULL, confirmed, off);
  }
  if (live && gl == 0 && ecs_done) {
#pragma unroll
    for (int k = 0; k < ECMC_NEV; ++k)
      if (cnt[k]) atomicAdd(&P.counters[k], cnt[k]);
    atomicAdd(&P.counters[CNT_EVENTS], nev_all);
    if (tried) atomicAdd(&P.counters[CNT_SWAP_TRIED], tried);
    if (confirmed) atomicAdd(&P.counters[CNT_CONFIRMED], confirmed);
    atomicAdd(&P.counters[CNT_ECS], ecs_done);
    atomicAdd(&P.sums[SUM_LIFT], lift_all);
    atomicAdd(&P.sums[SUM_REFL], refl_all);
    atomicAdd(&P.sums[SUM_DISP], disp_all);
  }

  // ------------------------------------------------------------ write back
  if (live) {
    for (int s = gl; s < m; s += G) {
      const int64_t b = st.id[s];
      Rr[3 * b] = st.px[s];
      Rr[3 * b + 1] = st.py[s];
      Rr[3 * b + 2] = st.pz[s];
    }
  }
}
#undef SYS

}  // namespace

size_t ec_smem_bytes(int stage_cap, int motile_cap, int ncell, int groups_per_block) {
  return (size_t)groups_per_block * group_bytes(stage_cap, motile_cap, motile_cap, ncell);
}

template <int G, bool F32, bool BATCH>
static cudaError_t launch_t(const ECParams &P, cudaStream_t s) {
  static int smem_max = 0;
  if (!smem_max) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
  }
  // whole warps per block (lockstep shuffles use all 32 lanes), at most 128
  // threads; among those, the block size that keeps the most groups (tiles)
  // resident per SM, as the occupancy calculator counts them
  const int per_warp = 32 / G;
  const int NC = P.domain ? (BATCH ? P.ncl_max : P.lg[0] * P.lg[1] * P.lg[2]) : 0;
  const int M = (F32 && P.domain) ? P.m_cap : P.stage_cap;
  const size_t per_group = ec_smem_bytes(P.stage_cap, M, NC, 1);
  const int need = (P.n_units + per_warp - 1) / per_warp * per_warp;
  static size_t memo_pg = 0;
  static int memo_need = 0, memo_gpb = 0;
  int gpb = 0, best = -1;
  const bool memo = memo_pg == per_group && memo_need == need;
  if (memo) {
    gpb = memo_gpb;
  } else {
    cudaError_t e = cudaFuncSetAttribute(ec_kernel<G, F32, BATCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return e;
  }
  for (int g = per_warp; !memo && g <= 128 / G; g += per_warp) {
    if ((size_t)g * per_group > (size_t)smem_max) break;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, ec_kernel<G, F32, BATCH>, g * G,
                                                      (size_t)g * per_group) != cudaSuccess)
      return cudaErrorInvalidValue;
    const int resident = blocks * (g < need ? g : need);
    if (resident >= best) {
      best = resident;
      gpb = g;
    }
    if (g >= need) break;
  }
  if (best >= 0) {
    memo_pg = per_group;
    memo_need = need;
    memo_gpb = gpb;
  }
  if (gpb == 0) return cudaErrorInvalidValue;
  const int threads = gpb * G;
  const size_t smem = (size_t)gpb * per_group;
  cudaError_t e = cudaFuncSetAttribute(ec_kernel<G, F32, BATCH>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (P.n_units + gpb - 1) / gpb;
  ec_kernel<G, F32, BATCH><<<blocks, threads, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_ec(const ECParams &P, int lanes, int fp32f, cudaStream_t s) {
  if (lanes == 32) return fp32f ? launch_t<32, true, false>(P, s) : launch_t<32, false, false>(P, s);
  if (lanes == 16) return fp32f ? launch_t<16, true, false>(P, s) : launch_t<16, false, false>(P, s);
  if (lanes == 8) return fp32f ? launch_t<8, true, false>(P, s) : launch_t<8, false, false>(P, s);
  if (lanes == 4) return fp32f ? launch_t<4, true, false>(P, s) : launch_t<4, false, false>(P, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_ec_batch(const ECParams &P, int lanes, int fp32f, cudaStream_t s) {
  if (lanes == 32) return fp32f ? launch_t<32, true, true>(P, s) : launch_t<32, false, true>(P, s);
  if (lanes == 16) return fp32f ? launch_t<16, true, true>(P, s) : launch_t<16, false, true>(P, s);
  if (lanes == 8) return fp32f ? launch_t<8, true, true>(P, s) : launch_t<8, false, true>(P, s);
  if (lanes == 4) return fp32f ? launch_t<4, true, true>(P, s) : launch_t<4, false, true>(P, s);
  return cudaErrorInvalidValue;
}

}  // namespace ecmc
