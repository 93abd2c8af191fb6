// C ABI and host orchestration of the EC library (declared in ecmc.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

using namespace ecmc;

namespace {
thread_local std::string g_err;

ecmc_status fail(ecmc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? ECMC_ENOMEM : ECMC_ECUDA,      \
                  "%s: %s", #call, cudaGetErrorString(e_));                         \
  } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (alloc_refused(sizeof(T) * count)) return cudaErrorMemoryAllocation;
  return cudaMalloc((void **)p, sizeof(T) * count);
}
}  // namespace

struct ecmc_ctx {
  int64_t n = 0;
  int32_t N = 1;
  double L[3] = {0, 0, 0};
  double sigma = 1.0, b_max = 1.2;
  ecmc_opts opts{};
  bool configured = false;
  // resolved run geometry
  double s_cap = 0.25, w = 1.2;
  double T[3] = {0, 0, 0}, W[3] = {0, 0, 0};
  double halo_hs = 0, halo_te = 0;
  int32_t nc[3] = {1, 1, 1};
  double cs[3] = {1, 1, 1};
  int64_t ncell = 1;
  int32_t stage_cap = 0;
  int32_t m_cap = 0;
  int32_t stage_tight = 0, m_tight = 0;  // block-lockstep first pass (0: one pass)
  int32_t *d_deferred = nullptr;         // units left to the second pass
  int64_t deferred_cap = 0;
  int32_t *d_n_deferred = nullptr;
  int32_t lanes = 32;
  // local cell grid of a tile (domain mode)
  int32_t lg[3] = {1, 1, 1};
  float linv[3] = {1, 1, 1};
  float lorg = 0.f;
  int64_t event_cap = 10000000;
  int32_t ecs_per_tile = 1;
  // stream
  cudaStream_t stream = nullptr;
  cudaStream_t own = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // device state
  double *d_r = nullptr;
  int32_t *d_img = nullptr;
  int32_t *d_tag = nullptr, *d_cell = nullptr, *d_rank = nullptr;
  int32_t *d_count = nullptr, *d_start = nullptr, *d_bsum = nullptr;
  double *d_cr = nullptr;
  float *d_crf = nullptr, *d_rf = nullptr;
  int32_t *d_cid = nullptr, *d_ctag = nullptr;
  int32_t *d_ftag = nullptr;  // final tags by bead (bead springs; on first use)
  unsigned long long *d_cnt = nullptr;
  double *d_sums = nullptr;
  int *d_status = nullptr;
  int32_t *d_unit_next = nullptr;
  double *d_obs_d = nullptr;
  unsigned long long *d_obs_u = nullptr;
  double *d_g1ref = nullptr;
  bool g1_set = false;
  // g1 table over log-spaced lags (ecmc_g1_track; allocated on first use)
  double *d_g1ring = nullptr, *d_g1sum = nullptr;
  unsigned long long *d_g1cnt = nullptr;
  size_t g1ring_n = 0;
  int32_t g1_P = 0, g1_K = 0;
  int64_t g1_t = 0;
  // chain structure scratch (allocated on first use)
  double *d_su = nullptr, *d_srec = nullptr, *d_spart = nullptr, *d_sr2n = nullptr;
  double *d_ssum = nullptr, *d_g2ref = nullptr;
  unsigned long long *d_shist = nullptr;
  int64_t shist_n = 0;
  // slow push-off: overlap flags and their count; a context made from
  // phantom chains may overlap until ecmc_pushoff has resolved it
  uint8_t *d_po_flag = nullptr;
  unsigned long long *d_po_cnt = nullptr;
  int64_t *d_po_ctr = nullptr;  // push-off: sweep index, sweeps run at this diameter
  bool pushoff_pending = false;
  // records
  uint64_t *d_rdig = nullptr;
  double *d_rlift = nullptr;
  int64_t *d_rev = nullptr;
  int64_t rec_cap = 0, rec_n = 0;
  ecmc_event *d_log = nullptr;
  unsigned long long *d_log_n = nullptr;
  int64_t log_cap = 0;
  // host counters
  int64_t sweeps_done = 0, ecs_done = 0;
  // counters, sweeps and ECs when the last ecmc_run started (d_cnt + CNT_N
  // holds that copy of the counters): ecmc_swap calibrates on that run
  int64_t mark_sweeps = 0, mark_ecs = 0;
  double device_seconds = 0.0;
  double ec_seconds = 0.0;
  std::vector<cudaEvent_t> kev;  // start/stop pairs around EC launches
};

namespace {

void free_cells(ecmc_ctx *c) {
  cudaFree(c->d_count);
  cudaFree(c->d_start);
  cudaFree(c->d_bsum);
  c->d_count = c->d_start = c->d_bsum = nullptr;
}

ecmc_status alloc_cells(ecmc_ctx *c) {
  free_cells(c);
  CU(dalloc(&c->d_count, c->ncell));
  CU(dalloc(&c->d_start, c->ncell + 1));
  CU(dalloc(&c->d_bsum, cells_scratch_ints(c->ncell)));
  return ECMC_OK;
}

// global cell grid of side >= cell_side (>= sigma), at least 3 per axis
ecmc_status set_grid(ecmc_ctx *c, double side) {
  int64_t ncell = 1;
  for (int a = 0; a < 3; ++a) {
    // bounded in double before the cast; the product stays below 2^31
    const double kd = floor(c->L[a] / side);
    if (!(kd >= 3.0)) return fail(ECMC_EINVAL, "box too small for the cell grid (axis %d)", a);
    if (!(kd <= 1048576.0) || (double)ncell * kd > 2147483647.0)
      return fail(ECMC_EINVAL, "cell grid too fine (axis %d)", a);
    const int k = (int)kd;
    c->nc[a] = k;
    c->cs[a] = c->L[a] / k;
    ncell *= k;
  }
  if (ncell != c->ncell || !c->d_count) {
    c->ncell = ncell;
    return alloc_cells(c);
  }
  return ECMC_OK;
}

CellParams cell_params(const ecmc_ctx *c, bool domain, uint64_t seed, int64_t sweep) {
  CellParams C{};
  C.n = c->n;
  for (int a = 0; a < 3; ++a) {
    C.L[a] = c->L[a];
    C.nc[a] = c->nc[a];
    C.cs[a] = c->cs[a];
    C.D[a] = c->opts.tiles[a];
    C.T[a] = c->T[a];
    C.W[a] = c->W[a];
  }
  C.domain = domain ? 1 : 0;
  C.seed = seed;
  C.replica = 0;
  C.sweep = sweep;
  C.r = c->d_r;
  C.tag = c->d_tag;
  C.cell = c->d_cell;
  C.rank = c->d_rank;
  C.count = c->d_count;
  C.start = c->d_start;
  C.block_sums = c->d_bsum;
  C.cr = c->d_cr;
  C.crf = c->d_crf;
  C.rf = c->d_rf;
  C.cid = c->d_cid;
  C.ctag = c->d_ctag;
  C.N = c->N;
  C.spring = (domain && c->configured && c->opts.k_spring > 0.0 && c->N > 1) ? 1 : 0;
  C.ftag = C.spring ? c->d_ftag : nullptr;
  return C;
}

ObsParams obs_params(const ecmc_ctx *c) {
  ObsParams O{};
  O.n = c->n;
  O.N = c->N;
  for (int a = 0; a < 3; ++a) {
    O.L[a] = c->L[a];
    O.half[a] = 0.5 * c->L[a];
    O.nc[a] = c->nc[a];
  }
  O.sig2 = c->sigma * c->sigma;
  O.b2 = c->b_max * c->b_max;
  O.r = c->d_r;
  O.img = c->d_img;
  O.g1ref = c->g1_set ? c->d_g1ref : nullptr;
  O.cr = c->d_cr;
  O.cid = c->d_cid;
  O.cstart = c->d_start;
  O.cell = c->d_cell;
  O.out_d = c->d_obs_d;
  O.out_u = c->d_obs_u;
  return O;
}

struct ObsHost {
  double re2_sum, bmax, bmin, g1_sum, bond_sum;
  unsigned long long overlaps, viol, pairs[2], taut[2];
};

// width of the contact shells (units of sigma)
constexpr double CONTACT_DELTA = 0.02;

// R_e^2, bonds, overlaps, g1 of the current positions (synchronises)
ecmc_status measure(ecmc_ctx *c, ObsHost *o) {
  // cells no narrower than the outer contact shell
  const double reach = (1.0 + 2.0 * CONTACT_DELTA) * c->sigma * (1.0 + 1e-9);
  double side = c->configured && c->opts.cell_side > 0 ? c->opts.cell_side : 1.05 * c->sigma;
  if (side < reach) side = reach;
  ecmc_status s = set_grid(c, side);
  if (s != ECMC_OK) return s;
  CU(launch_cells(cell_params(c, false, 0, 0), c->ncell, c->stream));
  const double init_d[5] = {0.0, 0.0, 1e300, 0.0, 0.0};
  CU(cudaMemcpyAsync(c->d_obs_d, init_d, sizeof(init_d), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemsetAsync(c->d_obs_u, 0, 6 * sizeof(unsigned long long), c->stream));
  ObsParams O = obs_params(c);
  {
    const double sg = c->sigma, bm = c->b_max, d = CONTACT_DELTA * c->sigma;
    O.c_lo = sg * sg * (1.0 - 1e-10);
    O.c_s1 = (sg + d) * (sg + d);
    O.c_s2 = (sg + 2.0 * d) * (sg + 2.0 * d);
    O.c_t0 = bm * bm * (1.0 + 1e-10);
    O.c_t1 = (bm - d) * (bm - d);
    O.c_t2 = (bm - 2.0 * d) * (bm - 2.0 * d);
  }
  CU(launch_obs(O, c->stream));
  double hd[5];
  unsigned long long hu[6];
  CU(cudaMemcpyAsync(hd, c->d_obs_d, sizeof(hd), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(hu, c->d_obs_u, sizeof(hu), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  o->re2_sum = hd[0];
  o->bmax = hd[1];
  o->bmin = c->N > 1 ? hd[2] : 0.0;
  o->g1_sum = hd[3];
  o->bond_sum = hd[4];
  o->overlaps = hu[0];
  o->viol = hu[1];
  o->pairs[0] = hu[2];
  o->pairs[1] = hu[3];
  o->taut[0] = hu[4];
  o->taut[1] = hu[5];
  return ECMC_OK;
}

ecmc_status check_state(ecmc_ctx *c) {
  ObsHost o;
  ecmc_status s = measure(c, &o);
  if (s != ECMC_OK) return s;
  if (o.overlaps) return fail(ECMC_EOVERLAP, "%llu overlapping pairs", o.overlaps);
  // (bead springs have no longest bond)
  const bool springs = c->configured && c->opts.k_spring > 0.0;
  if (o.viol && !springs) return fail(ECMC_ETETHER, "%llu bonds longer than b_max", o.viol);
  return ECMC_OK;
}

ecmc_status alloc_state(ecmc_ctx *c) {
  CU(dalloc(&c->d_r, 3 * c->n));
  CU(dalloc(&c->d_img, 3 * c->n));
  CU(cudaMemset(c->d_img, 0, sizeof(int32_t) * 3 * c->n));
  CU(dalloc(&c->d_tag, c->n));
  CU(dalloc(&c->d_cell, c->n));
  CU(dalloc(&c->d_rank, c->n));
  CU(dalloc(&c->d_cr, 3 * c->n));
  CU(dalloc(&c->d_crf, 3 * c->n));
  CU(dalloc(&c->d_rf, 3 * c->n));
  CU(dalloc(&c->d_cid, c->n));
  CU(dalloc(&c->d_ctag, c->n));
  CU(dalloc(&c->d_cnt, 2 * CNT_N));
  CU(cudaMemset(c->d_cnt, 0, sizeof(unsigned long long) * 2 * CNT_N));
  CU(dalloc(&c->d_sums, SUM_N));
  CU(cudaMemset(c->d_sums, 0, sizeof(double) * SUM_N));
  CU(dalloc(&c->d_status, 1));
  CU(cudaMemset(c->d_status, 0, sizeof(int)));
  CU(dalloc(&c->d_unit_next, 1));
  CU(dalloc(&c->d_n_deferred, 1));
  CU(dalloc(&c->d_obs_d, 5));
  CU(dalloc(&c->d_obs_u, 8));  // [6]: non-finite inputs of set_positions
  CU(dalloc(&c->d_g1ref, 3 * (c->n / c->N)));
  CU(cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking));
  c->stream = c->own;
  CU(cudaEventCreate(&c->ev0));
  CU(cudaEventCreate(&c->ev1));
  return ECMC_OK;
}

void destroy(ecmc_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  void *ptrs[] = {c->d_r, c->d_img, c->d_tag, c->d_cell, c->d_rank, c->d_count, c->d_start,
                  c->d_bsum, c->d_cr, c->d_crf, c->d_rf, c->d_cid, c->d_ctag, c->d_cnt, c->d_sums, c->d_status,
                  c->d_unit_next, c->d_n_deferred, c->d_ftag, c->d_deferred, c->d_obs_d, c->d_obs_u, c->d_g1ref, c->d_rdig, c->d_rlift, c->d_rev,
                  c->d_log, c->d_log_n, c->d_su, c->d_srec, c->d_spart,
                  c->d_sr2n, c->d_ssum, c->d_g2ref, c->d_shist, c->d_po_flag, c->d_po_cnt, c->d_po_ctr,
                  c->d_g1ring, c->d_g1sum, c->d_g1cnt};
  for (void *p : ptrs) cudaFree(p);
  for (cudaEvent_t e : c->kev) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

ecmc_status device_status(ecmc_ctx *c) {
  int st = 0;
  CU(cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (st == DEV_STUCK) return fail(ECMC_ESTUCK, "an event chain exceeded the event cap");
  if (st == DEV_CAPACITY) return fail(ECMC_ECAPACITY, "a tile exceeded the staging capacity");
  if (st == DEV_TILE) return fail(ECMC_ECAPACITY, "a bonded partner was not staged with its tile");
  if ((st & 0xFF) == DEV_BOUNDS)
    return fail(ECMC_EBOUNDS, "bounds-checked build: an index out of range was caught at site %d", st >> 8);
  return ECMC_OK;
}

ecmc_status make_ctx(const int32_t dims[3], double spacing, double jitter, uint64_t seed,
                     int32_t N, double sigma, double b_max, ecmc_ctx **out) {
  if (!out) return fail(ECMC_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dims || dims[0] < 1 || dims[1] < 1 || dims[2] < 1)
    return fail(ECMC_EINVAL, "lattice dims must be >= 1");
  if (!(sigma > 0.0)) return fail(ECMC_EINVAL, "sigma must be > 0");
  if (!(b_max >= sigma)) return fail(ECMC_EINVAL, "b_max must be >= sigma");
  if (N < 1) return fail(ECMC_EINVAL, "N must be >= 1");
  const int64_t n = (int64_t)dims[0] * dims[1] * dims[2];
  if (n % N) return fail(ECMC_EINVAL, "N must divide the number of sites");
  if (n >= (1ll << 29)) return fail(ECMC_EINVAL, "at most 2^29 beads");
  if (!(spacing >= sigma) || (N > 1 && !(spacing <= b_max)))
    return fail(ECMC_EINVAL, "need sigma <= spacing <= b_max");
  if (!(jitter >= 0.0) || !(2.0 * jitter < spacing - sigma + 1e-300) && jitter > 0.0)
    return fail(ECMC_EINVAL, "jitter must be in [0, (spacing - sigma)/2)");
  ecmc_ctx *c = new ecmc_ctx();
  c->n = n;
  c->N = N;
  for (int a = 0; a < 3; ++a) c->L[a] = dims[a] * spacing;
  c->sigma = sigma;
  c->b_max = b_max;
  ecmc_status s = alloc_state(c);
  if (s != ECMC_OK) {
    destroy(c);
    return s;
  }
  cudaError_t e = launch_lattice(dims, spacing, jitter, seed, 0, c->d_r, n, c->stream);
  if (e != cudaSuccess) {
    destroy(c);
    return fail(ECMC_ECUDA, "lattice: %s", cudaGetErrorString(e));
  }
  s = check_state(c);
  if (s != ECMC_OK) {
    destroy(c);
    return s;
  }
  *out = c;
  return ECMC_OK;
}

}  // namespace

namespace ecmc {
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace ecmc

extern "C" {

const char *ecmc_last_error(void) { return g_err.c_str(); }

ecmc_status ecmc_create_lattice(const int32_t dims[3], double spacing, double jitter,
                                uint64_t seed, int32_t N, double sigma, double b_max,
                                ecmc_ctx **out) {
  return make_ctx(dims, spacing, jitter, seed, N, sigma, b_max, out);
}

ecmc_status ecmc_create(const double box[3], double phi, int32_t n_chains, int32_t N,
                        double sigma, double b_max, ecmc_ctx **out) {
  if (!(phi > 0.0 && phi < 0.74)) return fail(ECMC_EINVAL, "phi must be in (0, 0.74)");
  if (n_chains < 1 || N < 1) return fail(ECMC_EINVAL, "n_chains and N must be >= 1");
  if (!(sigma > 0.0)) return fail(ECMC_EINVAL, "sigma must be > 0");
  const int64_t n = (int64_t)n_chains * N;
  const double vbead = M_PI * sigma * sigma * sigma / 6.0;
  double Lb[3];
  const bool given = box && (box[0] > 0.0 || box[1] > 0.0 || box[2] > 0.0);
  if (given) {
    if (!(box[0] > 0 && box[1] > 0 && box[2] > 0)) return fail(ECMC_EINVAL, "box must be > 0");
    const double phib = n * vbead / (box[0] * box[1] * box[2]);
    if (fabs(phib - phi) > 1e-3 * phi)
      return fail(ECMC_EINVAL, "box gives phi=%.6f, not %.6f", phib, phi);
    for (int a = 0; a < 3; ++a) Lb[a] = box[a];
  } else {
    const double side = cbrt(n * vbead / phi);
    Lb[0] = Lb[1] = Lb[2] = side;
  }
  // factor n into dims close to the box shape, all with the same spacing
  double best = 1e300;
  int32_t bd[3] = {0, 0, 0};
  const double a0 = cbrt(Lb[0] * Lb[1] * Lb[2] / (double)n);
  for (int64_t x = 1; x <= n && x <= 4096; ++x) {
    if (n % x) continue;
    const int64_t r = n / x;
    for (int64_t y = 1; y <= r && y <= 4096; ++y) {
      if (r % y) continue;
      const int64_t z = r / y;
      const double e = fabs(log(x * a0 / Lb[0])) + fabs(log(y * a0 / Lb[1])) + fabs(log(z * a0 / Lb[2]));
      if (e < best) {
        best = e;
        bd[0] = (int32_t)x;
        bd[1] = (int32_t)y;
        bd[2] = (int32_t)z;
      }
    }
  }
  if (!bd[0]) return fail(ECMC_EINVAL, "cannot factor n into a lattice");
  if (fabs(bd[0] * a0 - Lb[0]) > 1e-9 * Lb[0] || fabs(bd[1] * a0 - Lb[1]) > 1e-9 * Lb[1] ||
      fabs(bd[2] * a0 - Lb[2]) > 1e-9 * Lb[2]) {
    if (given) return fail(ECMC_EINVAL, "box shape does not fit a lattice of n sites");
  }
  return make_ctx(bd, a0, 0.01 * sigma, 0, N, sigma, b_max, out);
}

void ecmc_destroy(ecmc_ctx *ctx) { destroy(ctx); }

ecmc_status ecmc_set_stream(ecmc_ctx *c, void *stream) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  CU(cudaStreamSynchronize(c->stream));
  c->stream = stream ? (cudaStream_t)stream : c->own;
  return ECMC_OK;
}

ecmc_status ecmc_get_info(ecmc_ctx *c, double box[3], int64_t *n_beads, int32_t *N) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  if (box)
    for (int a = 0; a < 3; ++a) box[a] = c->L[a];
  if (n_beads) *n_beads = c->n;
  if (N) *N = c->N;
  return ECMC_OK;
}

ecmc_status ecmc_set_positions(ecmc_ctx *c, const double *xyz, const int32_t *img) {
  if (!c || !xyz) return fail(ECMC_EINVAL, "NULL argument");
  // copied as given (straight from pinned memory when the caller's buffers
  // are pinned), then wrapped and checked on the device
  CU(cudaMemcpyAsync(c->d_r, xyz, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice, c->stream));
  if (img)
    CU(cudaMemcpyAsync(c->d_img, img, sizeof(int32_t) * 3 * c->n, cudaMemcpyHostToDevice, c->stream));
  else
    CU(cudaMemsetAsync(c->d_img, 0, sizeof(int32_t) * 3 * c->n, c->stream));
  CU(cudaMemsetAsync(c->d_obs_u + 6, 0, sizeof(unsigned long long), c->stream));
  CU(launch_wrap(c->d_r, c->d_img, c->n, c->L, c->d_obs_u + 6, c->stream));
  unsigned long long bad = 0;
  CU(cudaMemcpyAsync(&bad, c->d_obs_u + 6, sizeof(bad), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->g1_set = false;
  if (bad) return fail(ECMC_EINVAL, "%llu non-finite coordinates", bad);
  ecmc_status st = check_state(c);
  if (st == ECMC_OK) c->pushoff_pending = false;
  return st;
}

ecmc_status ecmc_get_positions(ecmc_ctx *c, double *xyz, int32_t *img) {
  if (!c || !xyz) return fail(ECMC_EINVAL, "NULL argument");
  CU(cudaMemcpyAsync(xyz, c->d_r, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->stream));
  if (img) CU(cudaMemcpyAsync(img, c->d_img, sizeof(int32_t) * 3 * c->n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return ECMC_OK;
}

ecmc_status ecmc_configure(ecmc_ctx *c, const ecmc_opts *o) {
  if (!c || !o) return fail(ECMC_EINVAL, "NULL argument");
  ecmc_opts p = *o;
  if (p.mode != ECMC_MODE_SERIAL && p.mode != ECMC_MODE_DOMAIN) return fail(ECMC_EINVAL, "bad mode");
  if (p.dir_mode != ECMC_DIR_CART3 && p.dir_mode != ECMC_DIR_ISO) return fail(ECMC_EINVAL, "bad dir_mode");
  if (p.precision != ECMC_PREC_FP64 && p.precision != ECMC_PREC_FP32F)
    return fail(ECMC_EINVAL, "bad precision");
  const double sig = c->sigma;
  const double s_cap = p.s_cap > 0 ? p.s_cap : 0.25 * sig;
  const double w = p.joint > 0 ? p.joint : c->b_max;
  if (!(w >= c->b_max)) return fail(ECMC_EINVAL, "joint width must be >= b_max");
  const int lanes = p.lanes ? p.lanes : 32;
  if (lanes != 32 && lanes != 16 && lanes != 8 && lanes != 4)
    return fail(ECMC_EINVAL, "lanes must be 4, 8, 16 or 32");
  if (!(p.p_swap >= 0.0)) return fail(ECMC_EINVAL, "p_swap must be >= 0");
  if (!(p.k_spring >= 0.0 && p.k_spring < INFINITY)) return fail(ECMC_EINVAL, "k_spring must be finite and >= 0");
  if (p.k_spring > 0.0 && p.p_swap > 0.0)
    return fail(ECMC_EINVAL, "swaps are not defined for bead springs (p_swap must be 0)");
  if (p.schedule != 0 && p.schedule != 1) return fail(ECMC_EINVAL, "schedule must be 0 or 1");
  if (p.block_tiles < 0 || p.block_tiles > 32 || p.block_tiles * lanes > 128 ||
      (p.block_tiles > 0 && lanes > 1 && p.block_tiles % (32 / lanes) != 0))
    return fail(ECMC_EINVAL, "block_tiles must be a multiple of 32 / lanes, at most 32 and 128 / lanes");
  if (p.request_cap < 0 || p.request_cap > 6) return fail(ECMC_EINVAL, "request_cap must be in [0, 6]");
  if (!(p.tight_factor == 0.0 || (p.tight_factor >= 0.5 && p.tight_factor <= 4.0)))
    return fail(ECMC_EINVAL, "tight_factor must be 0 or in [0.5, 4]");
  const double margin = p.precision == ECMC_PREC_FP32F ? 0.01 * sig : 0.0;
  for (int a = 0; a < 3; ++a)
    if (!(s_cap + sig + margin < 0.5 * c->L[a])) return fail(ECMC_EINVAL, "need s_cap + sigma < L/2");
  const double halo_hs = sig * (1.0 + 1e-6);
  const double halo_te = (c->b_max > sig ? c->b_max : sig) * (1.0 + 1e-6);
  int32_t stage = p.stage_cap;
  int32_t mcap = 0;
  int32_t stage_t = 0, m_t = 0;
  if (p.mode == ECMC_MODE_DOMAIN) {
    for (int a = 0; a < 3; ++a) {
      if (p.tiles[a] < 3) return fail(ECMC_EINVAL, "tiles per axis must be >= 3");
      const double T = c->L[a] / p.tiles[a];
      const double W = T - w;
      if (!(W > 0.0)) return fail(ECMC_EINVAL, "tile narrower than the joint");
      if (!(W + 2.0 * halo_te < 0.5 * c->L[a]))
        return fail(ECMC_EINVAL, "tile plus halo must be < L/2 (use more tiles)");
      if (p.precision == ECMC_PREC_FP32F && !(W + 2.0 * halo_te <= 64.0 * sig))
        return fail(ECMC_EINVAL, "FP32 screen needs tiles of at most 64 sigma");
      c->T[a] = T;
      c->W[a] = W;
    }
    const double rho = (double)c->n / (c->L[0] * c->L[1] * c->L[2]);
    const double E[3] = {c->W[0] + 2.0 * halo_te, c->W[1] + 2.0 * halo_te, c->W[2] + 2.0 * halo_te};
    const bool derived = stage <= 0;
    if (derived) stage = stage_bound(E, rho);
    mcap = stage_bound(c->W, rho);
    if (derived) tight_caps(E, c->W, rho, stage, mcap, &stage_t, &m_t, p.tight_factor > 0 ? p.tight_factor : 1.08);
  } else {
    if (p.precision == ECMC_PREC_FP32F)
      for (int a = 0; a < 3; ++a)
        if (!(c->L[a] <= 64.0 * sig)) return fail(ECMC_EINVAL, "FP32 screen (serial) needs L <= 64 sigma");
    stage = (int32_t)c->n;
  }
  stage = (stage + 31) / 32 * 32;  // keeps the staging layouts 16-byte aligned
  if (stage > 65534) return fail(ECMC_EINVAL, "at most 65534 staged beads per tile (serial: beads)");
  int64_t ncl = 0;
  if (p.mode == ECMC_MODE_DOMAIN) {
    // local cell grid of a tile over [-h, W + h] with cells no narrower than
    // one free flight's reach (s_cap + 1.01 sigma) and than b_max
    const double hg = halo_te + 1e-3 * sig;
    const double reach = s_cap + sig + 0.01 * sig;
    const double bm = c->b_max * (1.0 + 1e-6);
    const double side_min = (reach > bm ? reach : bm) + 2e-3 * sig;
    ncl = 1;
    for (int a = 0; a < 3; ++a) {
      const double E = c->W[a] + 2.0 * hg;
      int g = (int)floor(E / side_min);
      if (g < 1) g = 1;
      c->lg[a] = g;
      c->linv[a] = (float)(g / E);
      ncl *= g;
    }
    c->lorg = (float)(-hg);
  }
  {
    int dev = 0, smem_max = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int gmin = 32 / lanes;
    if (mcap > stage) mcap = stage;
    const int M = (p.precision == ECMC_PREC_FP32F && p.mode == ECMC_MODE_DOMAIN) ? mcap : stage;
    const bool lock = p.mode == ECMC_MODE_DOMAIN && p.precision == ECMC_PREC_FP32F && p.schedule == 0 &&
                      p.k_spring == 0.0 && (lanes == 4 || lanes == 8 || lanes == 16);
    const int bt = p.block_tiles > 0 ? p.block_tiles : gmin;
    const size_t need = lock ? lock_smem_bytes(stage, M, (int)ncl, bt) : ec_smem_bytes(stage, M, (int)ncl, gmin);
    if ((int64_t)need > smem_max)
      return fail(ECMC_EINVAL, "staging needs %lld bytes of shared memory (max %d)",
                  (long long)need, smem_max);
  }
  c->opts = p;
  c->s_cap = s_cap;
  c->w = w;
  c->halo_hs = halo_hs;
  c->halo_te = halo_te;
  c->stage_cap = stage;
  c->m_cap = mcap > stage ? stage : mcap;
  c->stage_tight = stage_t;
  c->m_tight = m_t;
  if (p.mode == ECMC_MODE_DOMAIN) {
    const int64_t ntile = (int64_t)p.tiles[0] * p.tiles[1] * p.tiles[2];
    if (ntile > c->deferred_cap) {
      cudaFree(c->d_deferred);
      c->d_deferred = nullptr;
      c->deferred_cap = 0;
      CU(dalloc(&c->d_deferred, ntile));
      c->deferred_cap = ntile;
    }
  }
  c->lanes = lanes;
  c->event_cap = p.event_cap > 0 ? p.event_cap : 10000000;
  c->ecs_per_tile = p.ecs_per_tile > 0 ? p.ecs_per_tile : 1;
  c->configured = true;
  if (p.k_spring > 0.0 && p.mode == ECMC_MODE_DOMAIN && !c->d_ftag) CU(dalloc(&c->d_ftag, c->n));
  const double side = p.cell_side > 0 ? p.cell_side : 1.05 * sig;
  if (!(side >= sig)) return fail(ECMC_EINVAL, "cell side must be >= sigma");
  return set_grid(c, side);
}

ecmc_status ecmc_log_reserve(ecmc_ctx *c, int64_t cap) {
  if (!c || cap < 0) return fail(ECMC_EINVAL, "bad argument");
  cudaFree(c->d_log);
  cudaFree(c->d_log_n);
  c->d_log = nullptr;
  c->d_log_n = nullptr;
  c->log_cap = 0;
  if (cap > 0) {
    CU(dalloc(&c->d_log, cap));
    CU(dalloc(&c->d_log_n, 1));
    c->log_cap = cap;
  }
  return ECMC_OK;
}

static ecmc_status reserve_records(ecmc_ctx *c, int64_t units) {
  if (units <= c->rec_cap) return ECMC_OK;
  cudaFree(c->d_rdig);
  cudaFree(c->d_rlift);
  cudaFree(c->d_rev);
  c->d_rdig = nullptr;
  c->d_rlift = nullptr;
  c->d_rev = nullptr;
  c->rec_cap = 0;
  CU(dalloc(&c->d_rdig, units));
  CU(dalloc(&c->d_rlift, units));
  CU(dalloc(&c->d_rev, units));
  c->rec_cap = units;
  return ECMC_OK;
}

// one EC launch between a pair of events (the pair is reused across runs)
// the block-lockstep kernel runs the screened domain form with 4, 8 or 16 lanes
static bool uses_lock(const ecmc_opts &o, int lanes) {
  // (bead springs run in the warp-lockstep kernel)
  return o.mode == ECMC_MODE_DOMAIN && o.precision == ECMC_PREC_FP32F && o.schedule == 0 &&
         o.k_spring == 0.0 && (lanes == 4 || lanes == 8 || lanes == 16);
}

static cudaError_t timed_ec(ecmc_ctx *c, const ECParams &P, int64_t slot) {
  while ((int64_t)c->kev.size() < slot + 2) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    c->kev.push_back(e);
  }
  cudaError_t err = cudaEventRecord(c->kev[slot], c->stream);
  if (err != cudaSuccess) return err;
  if (uses_lock(c->opts, c->lanes)) err = launch_ec_lock(P, c->lanes, c->stream);
  else err = launch_ec(P, c->lanes, c->opts.precision == ECMC_PREC_FP32F, c->stream);
  if (err != cudaSuccess) return err;
  return cudaEventRecord(c->kev[slot + 1], c->stream);
}

static ECParams ec_params(const ecmc_ctx *c, uint64_t seed, double ell) {
  ECParams P{};
  P.block_tiles = c->opts.block_tiles;
  P.rq_per_tile = c->opts.request_cap > 0 ? c->opts.request_cap : 6;
  P.unit_next = c->d_unit_next;
  P.stage_tight = c->stage_tight;
  P.m_tight = c->m_tight;
  P.deferred = c->d_deferred;
  P.n_deferred = c->d_n_deferred;
  P.n = c->n;
  P.N = c->N;
  for (int a = 0; a < 3; ++a) {
    P.L[a] = c->L[a];
    P.half[a] = 0.5 * c->L[a];
    P.D[a] = c->opts.tiles[a];
    P.T[a] = c->T[a];
    P.W[a] = c->W[a];
    P.nc[a] = c->nc[a];
    P.cs[a] = c->cs[a];
  }
  P.sigma = c->sigma;
  P.sig2 = c->sigma * c->sigma;
  P.b2 = c->b_max * c->b_max;
  P.s_cap = c->s_cap;
  P.s_cap_f = round_up_f32(c->s_cap);
  P.domain = c->opts.mode == ECMC_MODE_DOMAIN;
  P.halo_hs = c->halo_hs;
  P.halo_te = c->halo_te;
  P.seed = seed;
  P.replica = 0;
  P.ell = ell;
  P.event_cap = c->event_cap;
  P.p_swap = c->opts.p_swap;
  P.swap_mode = c->opts.p_swap >= 1.0 ? 1 : (c->opts.p_swap > 0.0 ? 2 : 0);
  P.swap_thr = P.swap_mode == 2 ? (uint64_t)ceil(c->opts.p_swap * 9007199254740992.0) : 0;
  P.dir_mode = c->opts.dir_mode;
  P.stage_cap = c->stage_cap;
  P.m_cap = c->m_cap;
  // FP32 screen margins.  A shadow coordinate is off by at most
  // err = 2^-24 (3 L + 64 sigma) (FP32 rounding of the position, of the tile
  // corner, of their difference and of a wrap); a separation then by
  // 2 sqrt(3) err, d.v and |d|^2 - (d.v)^2 by about 3.5 err and 18 err.  The
  // margins keep a factor of 10 over those.
  {
    double Lm = c->L[0] > c->L[1] ? c->L[0] : c->L[1];
    Lm = Lm > c->L[2] ? Lm : c->L[2];
    const double err = (3.0 * Lm + 64.0 * c->sigma) / 16777216.0;
    const double ev = 35.0 * err > 2e-4 * c->sigma ? 35.0 * err : 2e-4 * c->sigma;
    const double ed = 180.0 * err * c->sigma > 1e-3 * c->sigma * c->sigma ? 180.0 * err * c->sigma
                                                                         : 1e-3 * c->sigma * c->sigma;
    P.eps_v = (float)ev;
    P.eps_d = (float)ed;
    P.eps_x = (float)ev;
  }
  for (int a = 0; a < 3; ++a) {
    P.lg[a] = c->lg[a];
    P.linv[a] = c->linv[a];
  }
  P.lorg = c->lorg;
  P.r = c->d_r;
  P.img = c->d_img;
  P.cr = c->d_cr;
  P.crf = c->d_crf;
  P.rf = c->d_rf;
  P.cid = c->d_cid;
  P.ctag = c->d_ctag;
  P.cstart = c->d_start;
  P.counters = c->d_cnt;
  P.sums = c->d_sums;
  P.status = c->d_status;
  P.k_spring = c->opts.k_spring;
  return P;
}

static G1Track g1_params(const ecmc_ctx *c) {
  G1Track G{};
  G.n = c->n;
  G.N = c->N;
  for (int a = 0; a < 3; ++a) G.L[a] = c->L[a];
  G.r = c->d_r;
  G.img = c->d_img;
  G.ring = c->d_g1ring;
  G.sum = c->d_g1sum;
  G.cnt = c->d_g1cnt;
  G.P = c->g1_P;
  G.K = c->g1_K;
  int64_t pk = 1;
  for (int k = 0; k < c->g1_K; ++k) {
    G.Pk[k] = pk;
    pk *= c->g1_P;
  }
  G.t = c->g1_t;
  return G;
}

// one sweep more of the g1 table (after the sweep's EC launch)
static cudaError_t g1_step(ecmc_ctx *c) {
  c->g1_t += 1;
  return launch_g1_track(g1_params(c), c->stream);
}

// copy the counters to the mark (d_cnt + CNT_N) in stream order and note the
// sweeps and ECs done
static cudaError_t mark_counters(ecmc_ctx *c) {
  c->mark_sweeps = c->sweeps_done;
  c->mark_ecs = c->ecs_done;
  return cudaMemcpyAsync(c->d_cnt + CNT_N, c->d_cnt, sizeof(unsigned long long) * CNT_N,
                         cudaMemcpyDeviceToDevice, c->stream);
}

ecmc_status ecmc_run(ecmc_ctx *c, double ell, int64_t chains_per_sweep, uint64_t seed,
                     int64_t n_sweeps) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  if (!c->configured) return fail(ECMC_EINVAL, "call ecmc_configure first");
  if (c->pushoff_pending) return fail(ECMC_EOVERLAP, "phantom chains overlap: run ecmc_pushoff first");
  if (!(ell >= 0.0) || !isfinite(ell)) return fail(ECMC_EINVAL, "ell must be finite and >= 0");
  const bool domain = c->opts.mode == ECMC_MODE_DOMAIN;
  const int64_t ntile = (int64_t)c->opts.tiles[0] * c->opts.tiles[1] * c->opts.tiles[2];
  const int k = domain ? (chains_per_sweep > 0 ? (int)chains_per_sweep : c->ecs_per_tile) : 1;
  int64_t units;
  if (domain) {
    if (n_sweeps < 0) return fail(ECMC_EINVAL, "n_sweeps must be >= 0");
    units = n_sweeps * ntile * k;
  } else {
    if (chains_per_sweep < 0) return fail(ECMC_EINVAL, "chains_per_sweep must be >= 0");
    units = chains_per_sweep;
  }
  CU(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  CU(mark_counters(c));
  ECParams P = ec_params(c, seed, ell);
  if (c->opts.record) {
    ecmc_status s = reserve_records(c, units);
    if (s != ECMC_OK) return s;
    CU(cudaMemsetAsync(c->d_rdig, 0, sizeof(uint64_t) * (units ? units : 1), c->stream));
    CU(cudaMemsetAsync(c->d_rlift, 0, sizeof(double) * (units ? units : 1), c->stream));
    CU(cudaMemsetAsync(c->d_rev, 0, sizeof(int64_t) * (units ? units : 1), c->stream));
    P.rec_digest = c->d_rdig;
    P.rec_lift = c->d_rlift;
    P.rec_events = c->d_rev;
    P.rec_cap = units;
    c->rec_n = units;
    if (c->d_log) {
      CU(cudaMemsetAsync(c->d_log_n, 0, sizeof(unsigned long long), c->stream));
      P.log = c->d_log;
      P.log_n = c->d_log_n;
      P.log_cap = c->log_cap;
    }
  }
  CU(cudaEventRecord(c->ev0, c->stream));
  if (domain) {
    P.n_units = (int32_t)ntile;
    P.ecs_per_tile = k;
    for (int64_t s = 0; s < n_sweeps; ++s) {
      const int64_t sweep = c->sweeps_done + s;
      CU(launch_cells(cell_params(c, true, seed, sweep), c->ncell, c->stream));
      P.sweep = sweep;
      P.rec_offset = s * ntile * k;
      CU(timed_ec(c, P, 2 * s));
      if (c->g1_P) CU(g1_step(c));
    }
  } else {
    P.n_units = 1;
    const int64_t chunk = 4096;
    for (int64_t j0 = 0; j0 < units; j0 += chunk) {
      const int64_t cnt = units - j0 < chunk ? units - j0 : chunk;
      P.sweep = c->ecs_done + j0;
      P.ecs_per_tile = (int32_t)cnt;
      P.rec_offset = j0;
      CU(timed_ec(c, P, 2 * (j0 / chunk)));
    }
  }
  CU(cudaEventRecord(c->ev1, c->stream));
  ecmc_status s = device_status(c);
  float ms = 0.f;
  CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->device_seconds += 1e-3 * ms;
  const int64_t launches = domain ? n_sweeps : (units + 4095) / 4096;
  for (int64_t i = 0; i < launches; ++i) {
    float kms = 0.f;
    CU(cudaEventElapsedTime(&kms, c->kev[2 * i], c->kev[2 * i + 1]));
    c->ec_seconds += 1e-3 * kms;
  }
  if (domain) c->sweeps_done += n_sweeps;
  else c->ecs_done += units;
  return s;
}

ecmc_status ecmc_swap(ecmc_ctx *c, double target) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  if (!(target >= 0.0)) return fail(ECMC_EINVAL, "target must be >= 0");
  if (target == 0.0) {
    c->opts.p_swap = 0.0;
    return ECMC_OK;
  }
  // the motile contacts and sweeps of the last ecmc_run call
  unsigned long long h[2 * CNT_N];
  CU(cudaMemcpyAsync(h, c->d_cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const unsigned long long *m = h + CNT_N;
  const double contacts = (double)((h[ECMC_EV_HS_LIFT] - m[ECMC_EV_HS_LIFT]) + (h[ECMC_EV_SWAP] - m[ECMC_EV_SWAP]));
  const double sweeps = c->opts.mode == ECMC_MODE_DOMAIN
                            ? (double)(c->sweeps_done - c->mark_sweeps)
                            : (double)(c->ecs_done - c->mark_ecs) / (double)c->n;
  if (!(contacts > 0.0) || !(sweeps > 0.0))
    return fail(ECMC_EINVAL, "run EC sweeps (ecmc_run) before calibrating swaps");
  double p = target * (double)c->n * sweeps / contacts;
  c->opts.p_swap = p > 1.0 ? 1.0 : p;
  return ECMC_OK;
}

ecmc_status ecmc_observables(ecmc_ctx *c, ecmc_obs *out) {
  if (!c || !out) return fail(ECMC_EINVAL, "NULL argument");
  ObsHost o;
  ecmc_status s = measure(c, &o);
  if (s != ECMC_OK) return s;
  unsigned long long h[CNT_N];
  double sums[SUM_N];
  CU(cudaMemcpyAsync(h, c->d_cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(sums, c->d_sums, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof(*out));
  out->n_beads = c->n;
  out->n_chains = c->n / c->N;
  out->N = c->N;
  out->sweeps = c->sweeps_done;
  out->ecs = (int64_t)h[CNT_ECS];
  for (int k = 0; k < ECMC_NEV; ++k) out->events[k] = (int64_t)h[k];
  out->events_total = (int64_t)h[CNT_EVENTS];
  out->swap_tried = (int64_t)h[CNT_SWAP_TRIED];
  out->lift_sum = sums[SUM_LIFT];
  out->refl_sum = sums[SUM_REFL];
  out->disp_sum = sums[SUM_DISP];  // ell summed per EC (the flights add up to it)
  out->ell_sum = sums[SUM_DISP];
  out->pressure = out->ell_sum > 0 ? 1.0 + out->lift_sum / out->ell_sum : 0.0;
  out->re2_mean = o.re2_sum / (double)(c->n / c->N);
  out->bond_max = o.bmax;
  out->bond_min = o.bmin;
  out->overlaps = (int64_t)o.overlaps;
  out->tether_violations = (int64_t)o.viol;
  out->g1 = c->g1_set ? o.g1_sum / (double)(c->n / c->N) : 0.0;
  out->device_seconds = c->device_seconds;
  out->ec_kernel_seconds = c->ec_seconds;
  out->confirmed = (int64_t)h[CNT_CONFIRMED];
  out->exhaustive = (int64_t)h[CNT_EXHAUSTIVE];
  out->bond_mean = c->N > 1 ? o.bond_sum / (double)((c->n / c->N) * (c->N - 1)) : 0.0;
  const double d = CONTACT_DELTA * c->sigma;
  for (int k = 0; k < 2; ++k) {
    out->contact_pairs[k] = (int64_t)o.pairs[k];
    out->taut_bonds[k] = (int64_t)o.taut[k];
  }
  out->contact_delta = d;
  const double fs = (1.5 * (double)o.pairs[0] - 0.5 * (double)o.pairs[1]) / d;
  const double fb = (1.5 * (double)o.taut[0] - 0.5 * (double)o.taut[1]) / d;
  out->pressure_contact = 1.0 + (c->sigma * fs - c->b_max * fb) / (3.0 * (double)c->n);
  return ECMC_OK;
}

// the chain-structure pass over the current positions (scratch on demand)
static ecmc_status run_structure(ecmc_ctx *c, bool with_r2n, double dR, int64_t nbins) {
  const int64_t nch = c->n / c->N;
  if (!c->d_su) {
    CU(dalloc(&c->d_su, 3 * c->n));
    CU(dalloc(&c->d_srec, STRUCT_REC * nch));
    CU(dalloc(&c->d_ssum, STRUCT_SUMS));
    CU(dalloc(&c->d_g2ref, 3 * nch));
  }
  if (with_r2n && !c->d_spart) {
    CU(dalloc(&c->d_spart, nch * c->N));
    CU(dalloc(&c->d_sr2n, c->N));
  }
  if (nbins > c->shist_n) {
    cudaFree(c->d_shist);
    c->d_shist = nullptr;
    c->shist_n = 0;
    CU(cudaMalloc(&c->d_shist, sizeof(unsigned long long) * (size_t)nbins));
    c->shist_n = nbins;
  }
  StructParams S{};
  S.n = c->n;
  S.N = c->N;
  for (int a = 0; a < 3; ++a) {
    S.L[a] = c->L[a];
    S.half[a] = 0.5 * c->L[a];
  }
  S.r = c->d_r;
  S.u = c->d_su;
  S.rec = c->d_srec;
  S.mref = c->g1_set ? c->d_g2ref : nullptr;
  S.part = with_r2n ? c->d_spart : nullptr;
  S.r2n = with_r2n ? c->d_sr2n : nullptr;
  S.sums = c->d_ssum;
  S.hist = nbins > 0 ? c->d_shist : nullptr;
  S.nbins = nbins;
  S.dR = dR;
  CU(launch_struct(S, c->stream));
  return ECMC_OK;
}

ecmc_status ecmc_phantom_chains(const double L[3], int64_t n_chains, int32_t N, double bond,
                                double c, uint64_t seed, double *xyz_out, int32_t *img_out) {
  if (!L || !xyz_out) return fail(ECMC_EINVAL, "NULL argument");
  for (int a = 0; a < 3; ++a)
    if (!(L[a] > 0.0 && L[a] < INFINITY)) return fail(ECMC_EINVAL, "box must be positive and finite");
  if (n_chains < 1 || N < 1 || n_chains > ((int64_t)1 << 40) / N)
    return fail(ECMC_EINVAL, "need n_chains >= 1, N >= 1 and at most 2^40 beads");
  if (!(bond > 0.0 && bond < INFINITY)) return fail(ECMC_EINVAL, "bond must be positive");
  if (!(c >= 1.0 && c < INFINITY)) return fail(ECMC_EINVAL, "stiffness c must be >= 1");
  const int64_t n = n_chains * N;
  double *d_r = nullptr;
  int32_t *d_img = nullptr;
  unsigned long long *d_bad = nullptr;
  cudaError_t e = cudaMalloc(&d_r, sizeof(double) * 3 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_img, sizeof(int32_t) * 3 * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, sizeof(unsigned long long) * 2);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_img, 0, sizeof(int32_t) * 3 * (size_t)n, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long) * 2, 0);
  const double ct = (c - 3.0) / (c + 1.0);
  if (e == cudaSuccess) e = launch_phantom(n_chains, N, L, bond, ct, seed, d_r, d_bad, 0);
  if (e == cudaSuccess) e = launch_wrap(d_r, d_img, n, L, d_bad + 1, 0);
  unsigned long long bad[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(xyz_out, d_r, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && img_out)
    e = cudaMemcpy(img_out, d_img, sizeof(int32_t) * 3 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d_r);
  cudaFree(d_img);
  cudaFree(d_bad);
  if (e != cudaSuccess) return fail(ECMC_ECUDA, "%s", cudaGetErrorString(e));
  if (bad[0] || bad[1]) return fail(ECMC_EINVAL, "phantom walk failed (%llu walks, %llu coordinates)", bad[0], bad[1]);
  return ECMC_OK;
}

ecmc_status ecmc_create_phantom(const double box[3], int64_t n_chains, int32_t N, double bond,
                                double stiffness, uint64_t seed, double sigma, double b_max,
                                ecmc_ctx **out) {
  if (!out || !box) return fail(ECMC_EINVAL, "NULL argument");
  *out = nullptr;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0.0 && box[a] < INFINITY)) return fail(ECMC_EINVAL, "box must be positive and finite");
  if (n_chains < 1 || N < 1 || n_chains >= ((int64_t)1 << 29) / N)
    return fail(ECMC_EINVAL, "need n_chains >= 1, N >= 1 and fewer than 2^29 beads");
  if (!(sigma > 0.0)) return fail(ECMC_EINVAL, "sigma must be > 0");
  if (!(b_max >= sigma)) return fail(ECMC_EINVAL, "b_max must be >= sigma");
  if (!(bond > 0.0 && bond <= b_max)) return fail(ECMC_EINVAL, "bond must be in (0, b_max]");
  if (!(stiffness >= 1.0 && stiffness < INFINITY)) return fail(ECMC_EINVAL, "stiffness c must be >= 1");
  ecmc_ctx *c = new ecmc_ctx();
  c->n = n_chains * N;
  c->N = N;
  for (int a = 0; a < 3; ++a) c->L[a] = box[a];
  c->sigma = sigma;
  c->b_max = b_max;
  ecmc_status s = alloc_state(c);
  if (s != ECMC_OK) {
    destroy(c);
    return s;
  }
  const double ct = (stiffness - 3.0) / (stiffness + 1.0);
  unsigned long long bad[2] = {0, 0};
  cudaError_t e = cudaMemsetAsync(c->d_obs_u + 6, 0, 2 * sizeof(unsigned long long), c->stream);
  if (e == cudaSuccess) e = launch_phantom(n_chains, N, c->L, bond, ct, seed, c->d_r, c->d_obs_u + 6, c->stream);
  if (e == cudaSuccess) e = launch_wrap(c->d_r, c->d_img, c->n, c->L, c->d_obs_u + 7, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bad, c->d_obs_u + 6, sizeof(bad), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess || bad[0] || bad[1]) {
    destroy(c);
    if (e != cudaSuccess) return fail(ECMC_ECUDA, "phantom chains: %s", cudaGetErrorString(e));
    return fail(ECMC_EINVAL, "phantom walk failed");
  }
  c->pushoff_pending = true;
  *out = c;
  return ECMC_OK;
}

ecmc_status ecmc_pushoff(ecmc_ctx *c, double f0, int32_t stages, double ell, uint64_t seed,
                         int64_t max_sweeps, int64_t *sweeps_out) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  if (sweeps_out) *sweeps_out = 0;
  if (!c->configured || c->opts.mode != ECMC_MODE_DOMAIN || c->opts.precision != ECMC_PREC_FP64)
    return fail(ECMC_EINVAL, "push-off needs the domain mode and FP64");
  if (!(f0 > 0.0 && f0 <= 1.0) || stages < 1 || max_sweeps < 1 || !(ell >= 0.0 && ell < INFINITY))
    return fail(ECMC_EINVAL, "need 0 < f0 <= 1, stages >= 1, max_sweeps >= 1, finite ell >= 0");
  if (!c->d_po_flag) {
    CU(dalloc(&c->d_po_flag, c->n));
    CU(dalloc(&c->d_po_cnt, 1));
    CU(dalloc(&c->d_po_ctr, 2));
  }
  CU(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  ECParams P = ec_params(c, seed, ell);
  const int64_t ntile = (int64_t)c->opts.tiles[0] * c->opts.tiles[1] * c->opts.tiles[2];
  P.n_units = (int32_t)ntile;
  P.ecs_per_tile = 1;
  P.swap_mode = 0;
  P.p_swap = 0.0;
  P.po_flag = c->d_po_flag;
  {
    // phantom chains are far more clustered than a melt (a tile's content
    // varies about three times as much): stage up to 2.5 times the mean
    // content plus 64 (capacities change no event)
    const double rho = (double)c->n / (c->L[0] * c->L[1] * c->L[2]);
    double vol = 1.0;
    for (int a = 0; a < 3; ++a) vol *= c->W[a] + 2.0 * c->halo_te;
    int64_t S = (int64_t)ceil(2.5 * rho * vol + 64.0);
    S = (S + 31) / 32 * 32;
    if (S < c->stage_cap) S = c->stage_cap;
    if (S > 65504) S = 65504;
    int dev = 0, smem_max = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int ncl = c->lg[0] * c->lg[1] * c->lg[2];
    if (ec_smem_bytes((int)S, (int)S, ncl, 32 / c->lanes) > (size_t)smem_max)
      return fail(ECMC_EINVAL, "push-off staging of %lld beads per tile does not fit in shared memory "
                  "(use smaller tiles or more lanes)", (long long)S);
    P.stage_cap = (int32_t)S;
    P.m_cap = (int32_t)S;
  }
  // The sweeps run from the device: the sweep index and the sweeps run at
  // the current diameter live in d_po_ctr; every sweep is the cell pass,
  // the overlap flags and an EC launch that does nothing once no bead
  // overlaps, then the counters advance only if that launch ran.  The host
  // reads the counters once per chunk of sweeps (and checks the flags once
  // more after it), so a stage that ends inside a chunk ends exactly where
  // the sweep-by-sweep loop would.
  const ObsParams O = obs_params(c);
  P.sweep_dev = c->d_po_ctr;
  P.po_count = c->d_po_cnt;
  const int64_t CHUNK = 64;
  int64_t sweeps = 0;
  int64_t ctr[2] = {c->sweeps_done, 0};
  CU(cudaMemcpyAsync(c->d_po_ctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice, c->stream));
  CellParams C = cell_params(c, true, seed, 0);
  C.sweep_dev = c->d_po_ctr;
  for (int32_t k = 0; k <= stages; ++k) {
    const double d =
        k == stages ? c->sigma : c->sigma * (f0 + (1.0 - f0) * (double)k / (double)stages);
    P.sigma = d;
    P.sig2 = d * d;
    const double thr = d * d * (1.0 - 1e-10);
    CU(cudaMemsetAsync(c->d_po_ctr + 1, 0, sizeof(int64_t), c->stream));
    int64_t ran = 0;
    for (;;) {
      const int64_t n = max_sweeps - ran < CHUNK ? max_sweeps - ran : CHUNK;
      for (int64_t i = 0; i < n; ++i) {
        CU(launch_cells(C, c->ncell, c->stream));
        CU(launch_po_flags(O, thr, c->d_po_flag, c->d_po_cnt, c->stream));
        CU(launch_ec(P, c->lanes, 0, c->stream));
        CU(launch_po_advance(c->d_po_cnt, c->d_po_ctr, c->stream));
      }
      // the overlaps left after the chunk
      CU(launch_cells(C, c->ncell, c->stream));
      CU(launch_po_flags(O, thr, c->d_po_flag, c->d_po_cnt, c->stream));
      unsigned long long cnt = 0;
      CU(cudaMemcpyAsync(&cnt, c->d_po_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
      CU(cudaMemcpyAsync(ctr, c->d_po_ctr, sizeof(ctr), cudaMemcpyDeviceToHost, c->stream));
      ecmc_status st = device_status(c);  // synchronises
      if (st != ECMC_OK) return st;
      ran = ctr[1];
      c->sweeps_done = ctr[0];
      if (cnt == 0) break;
      if (ran >= max_sweeps) {
        if (sweeps_out) *sweeps_out = sweeps + ran;
        return fail(ECMC_ESTUCK, "push-off: %llu beads overlap at diameter %.6g after %lld sweeps",
                    cnt, d, (long long)max_sweeps);
      }
    }
    sweeps += ran;
  }
  if (sweeps_out) *sweeps_out = sweeps;
  CU(mark_counters(c));  // push-off sweeps are no run to calibrate swaps on
  ecmc_status st = check_state(c);
  if (st == ECMC_OK) c->pushoff_pending = false;
  return st;
}

ecmc_status ecmc_g1_reset(ecmc_ctx *c) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  CU(launch_g1_snapshot(obs_params(c), c->d_g1ref, c->stream));
  if (c->N >= 2) {
    // g2 reference: the middle beads relative to their centre of mass
    const bool had = c->g1_set;
    c->g1_set = false;
    ecmc_status st = run_structure(c, false, 1.0, 0);
    c->g1_set = had;
    if (st != ECMC_OK) return st;
    CU(cudaMemcpy2DAsync(c->d_g2ref, 3 * sizeof(double), c->d_srec + 10, STRUCT_REC * sizeof(double),
                         3 * sizeof(double), (size_t)(c->n / c->N), cudaMemcpyDeviceToDevice,
                         c->stream));
  }
  c->g1_set = true;
  CU(cudaStreamSynchronize(c->stream));
  return ECMC_OK;
}

ecmc_status ecmc_g1_track(ecmc_ctx *c, int32_t P, int32_t K) {
  if (!c) return fail(ECMC_EINVAL, "ctx is NULL");
  if (P == 0) {
    c->g1_P = 0;
    return ECMC_OK;
  }
  if (P < 2 || P > 64 || K < 1 || K > 16) return fail(ECMC_EINVAL, "need 2 <= P <= 64 and 1 <= K <= 16");
  double top = 1.0;
  for (int k = 0; k < K; ++k) top *= P;
  if (!(top < 4.0e18)) return fail(ECMC_EINVAL, "P^K must stay below 4e18 sweeps");
  const int64_t nch = c->n / c->N;
  const size_t ring_n = (size_t)K * P * (size_t)nch * 3;
  const size_t nlag = (size_t)K * (P - 1);
  if (ring_n > c->g1ring_n) {
    cudaFree(c->d_g1ring);
    c->d_g1ring = nullptr;
    c->g1ring_n = 0;
    CU(dalloc(&c->d_g1ring, ring_n));
    c->g1ring_n = ring_n;
  }
  if (!c->d_g1sum) {
    CU(dalloc(&c->d_g1sum, 16 * 63));
    CU(dalloc(&c->d_g1cnt, 16 * 63));
  }
  CU(cudaMemsetAsync(c->d_g1sum, 0, sizeof(double) * nlag, c->stream));
  CU(cudaMemsetAsync(c->d_g1cnt, 0, sizeof(unsigned long long) * nlag, c->stream));
  c->g1_P = P;
  c->g1_K = K;
  c->g1_t = 0;
  CU(launch_g1_track(g1_params(c), c->stream));  // the snapshot at t = 0
  return ECMC_OK;
}

ecmc_status ecmc_g1_table(ecmc_ctx *c, int64_t *lag, double *g1, int64_t *count, int32_t cap,
                          int32_t *n) {
  if (!c || !n) return fail(ECMC_EINVAL, "NULL argument");
  if (!c->d_g1sum || c->g1_K == 0) {
    *n = 0;
    return ECMC_OK;
  }
  const int nlag = c->g1_K * (c->g1_P - 1);
  std::vector<double> sum((size_t)nlag);
  std::vector<unsigned long long> cnt((size_t)nlag);
  CU(cudaMemcpyAsync(sum.data(), c->d_g1sum, sizeof(double) * nlag, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(cnt.data(), c->d_g1cnt, sizeof(unsigned long long) * nlag, cudaMemcpyDeviceToHost,
                     c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const int m = nlag < cap ? nlag : (cap > 0 ? cap : 0);
  const double nch = (double)(c->n / c->N);
  int64_t pk = 1;
  for (int k = 0, q = 0; k < c->g1_K; ++k, pk *= c->g1_P) {
    for (int j = 1; j < c->g1_P; ++j, ++q) {
      if (q >= m) break;
      if (lag) lag[q] = (int64_t)j * pk;
      if (count) count[q] = (int64_t)cnt[q];
      if (g1) g1[q] = cnt[q] ? sum[q] / ((double)cnt[q] * nch) : 0.0;
    }
  }
  *n = m;
  return ECMC_OK;
}

ecmc_status ecmc_structure(ecmc_ctx *c, ecmc_struct *out, double *r2n, double dR, int64_t nbins,
                           int64_t *hist) {
  if (!c || !out) return fail(ECMC_EINVAL, "NULL argument");
  if (c->N < 2) return fail(ECMC_EINVAL, "chain structure needs chains of at least 2 beads");
  if (nbins < 0 || (nbins > 0 && !hist)) return fail(ECMC_EINVAL, "nbins must be >= 0 with a histogram buffer");
  if (!hist) nbins = 0;
  if (nbins > 0 && !(dR > 0.0 && dR < INFINITY)) return fail(ECMC_EINVAL, "dR must be positive and finite");
  ecmc_status st = run_structure(c, r2n != nullptr, dR, nbins);
  if (st != ECMC_OK) return st;
  double sums[STRUCT_SUMS];
  CU(cudaMemcpyAsync(sums, c->d_ssum, sizeof(sums), cudaMemcpyDeviceToHost, c->stream));
  if (r2n) CU(cudaMemcpyAsync(r2n, c->d_sr2n, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  std::vector<unsigned long long> h((size_t)nbins);
  if (nbins > 0)
    CU(cudaMemcpyAsync(h.data(), c->d_shist, sizeof(unsigned long long) * (size_t)nbins,
                       cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  for (int64_t b = 0; b < nbins; ++b) hist[b] = (int64_t)h[(size_t)b];
  memset(out, 0, sizeof(*out));
  out->n_chains = c->n / c->N;
  out->N = c->N;
  out->rg2_sum = sums[0];
  for (int k = 0; k < 3; ++k) out->lam_sum[k] = sums[1 + k];
  out->b_sum = sums[4];
  out->c_sum = sums[5];
  out->kappa2_sum = sums[6];
  out->bc_sum = sums[7];
  out->g2_sum = c->g1_set ? sums[8] : 0.0;
  out->re2_sum = sums[9];
  return ECMC_OK;
}

ecmc_status ecmc_records(ecmc_ctx *c, uint64_t *digest, double *lift, int64_t *events,
                         int64_t *n) {
  if (!c || !n) return fail(ECMC_EINVAL, "NULL argument");
  if (!c->d_rdig) {
    *n = 0;
    return ECMC_OK;
  }
  const int64_t cnt = c->rec_n < *n ? c->rec_n : *n;
  if (digest) CU(cudaMemcpyAsync(digest, c->d_rdig, sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, c->stream));
  if (lift) CU(cudaMemcpyAsync(lift, c->d_rlift, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream));
  if (events) CU(cudaMemcpyAsync(events, c->d_rev, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  *n = cnt;
  return ECMC_OK;
}

ecmc_status ecmc_event_log(ecmc_ctx *c, ecmc_event *buf, int64_t cap, int64_t *n) {
  if (!c || !n) return fail(ECMC_EINVAL, "NULL argument");
  if (!c->d_log) {
    *n = 0;
    return ECMC_OK;
  }
  unsigned long long used = 0;
  CU(cudaMemcpyAsync(&used, c->d_log_n, sizeof(used), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  int64_t cnt = (int64_t)used;
  if (cnt > c->log_cap) cnt = c->log_cap;
  if (cnt > cap) cnt = cap;
  if (buf && cnt > 0)
    CU(cudaMemcpyAsync(buf, c->d_log, sizeof(ecmc_event) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  *n = cnt;
  return ECMC_OK;
}

ecmc_status ecmc_domain_tags(ecmc_ctx *c, uint64_t seed, int64_t sweep, int32_t *tags,
                             double shift[3]) {
  if (!c || !tags) return fail(ECMC_EINVAL, "NULL argument");
  if (!c->configured || c->opts.mode != ECMC_MODE_DOMAIN)
    return fail(ECMC_EINVAL, "configure the domain mode first");
  CU(launch_cells(cell_params(c, true, seed, sweep), c->ncell, c->stream));
  CU(cudaMemcpyAsync(tags, (c->opts.k_spring > 0.0 && c->N > 1) ? c->d_ftag : c->d_tag, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (shift) {
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)sweep, 0, 0, seed, 0);
    for (int a = 0; a < 3; ++a) shift[a] = unit53(w.v[a]) * c->T[a];
  }
  return ECMC_OK;
}

// ---------------------------------------------------------------- checkpoint
namespace {
const uint64_t CKPT_MAGIC = 0x45434D434B505431ull;  // "ECMCKPT1"
struct CkptHeader {
  uint64_t magic;
  uint32_t version;
  uint32_t pad;
  int64_t n;
  int32_t N;
  int32_t pad2;
  double L[3];
  double sigma, b_max;
  int64_t sweeps_done, ecs_done;
  double device_seconds;
  uint64_t counters[CNT_N];
  double sums[SUM_N];
  ecmc_opts opts;
  int32_t configured;
  int32_t pad3;
};
uint64_t checksum(const void *p, size_t len, uint64_t h) {
  const unsigned char *b = (const unsigned char *)p;
  for (size_t i = 0; i < len; ++i) {
    h ^= b[i];
    h *= 0x100000001B3ull;
  }
  return h;
}
}  // namespace

ecmc_status ecmc_checkpoint(ecmc_ctx *c, const char *path) {
  if (!c || !path) return fail(ECMC_EINVAL, "NULL argument");
  CkptHeader hd;
  memset(&hd, 0, sizeof(hd));
  hd.magic = CKPT_MAGIC;
  hd.version = 3;
  hd.n = c->n;
  hd.N = c->N;
  for (int a = 0; a < 3; ++a) hd.L[a] = c->L[a];
  hd.sigma = c->sigma;
  hd.b_max = c->b_max;
  hd.sweeps_done = c->sweeps_done;
  hd.ecs_done = c->ecs_done;
  hd.device_seconds = c->device_seconds;
  hd.opts = c->opts;
  hd.configured = c->configured;
  std::vector<double> r(3 * c->n);
  std::vector<int32_t> im(3 * c->n);
  CU(cudaMemcpyAsync(hd.counters, c->d_cnt, sizeof(hd.counters), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(hd.sums, c->d_sums, sizeof(hd.sums), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(r.data(), c->d_r, sizeof(double) * r.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(im.data(), c->d_img, sizeof(int32_t) * im.size(), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  uint64_t h = 0xCBF29CE484222325ull;
  h = checksum(&hd, sizeof(hd), h);
  h = checksum(r.data(), sizeof(double) * r.size(), h);
  h = checksum(im.data(), sizeof(int32_t) * im.size(), h);
  FILE *f = fopen(path, "wb");
  if (!f) return fail(ECMC_ECKPT, "cannot open %s", path);
  bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 &&
            fwrite(r.data(), sizeof(double), r.size(), f) == r.size() &&
            fwrite(im.data(), sizeof(int32_t), im.size(), f) == im.size() &&
            fwrite(&h, sizeof(h), 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(ECMC_ECKPT, "write failed: %s", path);
  return ECMC_OK;
}

ecmc_status ecmc_restore(ecmc_ctx *c, const char *path) {
  if (!c || !path) return fail(ECMC_EINVAL, "NULL argument");
  FILE *f = fopen(path, "rb");
  if (!f) return fail(ECMC_ECKPT, "cannot open %s", path);
  CkptHeader hd;
  std::vector<double> r(3 * c->n);
  std::vector<int32_t> im(3 * c->n);
  uint64_t hfile = 0;
  bool ok = fread(&hd, sizeof(hd), 1, f) == 1;
  ok = ok && hd.magic == CKPT_MAGIC && hd.version == 3 && hd.n == c->n && hd.N == c->N;
  ok = ok && fread(r.data(), sizeof(double), r.size(), f) == r.size() &&
       fread(im.data(), sizeof(int32_t), im.size(), f) == im.size() &&
       fread(&hfile, sizeof(hfile), 1, f) == 1;
  fclose(f);
  if (!ok) return fail(ECMC_ECKPT, "checkpoint does not match this context");
  uint64_t h = 0xCBF29CE484222325ull;
  h = checksum(&hd, sizeof(hd), h);
  h = checksum(r.data(), sizeof(double) * r.size(), h);
  h = checksum(im.data(), sizeof(int32_t) * im.size(), h);
  if (h != hfile) return fail(ECMC_ECKPT, "checkpoint checksum mismatch");
  for (int a = 0; a < 3; ++a)
    if (hd.L[a] != c->L[a]) return fail(ECMC_ECKPT, "box differs");
  CU(cudaMemcpyAsync(c->d_r, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_img, im.data(), sizeof(int32_t) * im.size(), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_cnt, hd.counters, sizeof(hd.counters), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_sums, hd.sums, sizeof(hd.sums), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  c->sweeps_done = hd.sweeps_done;
  c->ecs_done = hd.ecs_done;
  c->device_seconds = hd.device_seconds;
  CU(mark_counters(c));
  if (hd.configured) return ecmc_configure(c, &hd.opts);
  return ECMC_OK;
}

ecmc_status ecmc_autotune(ecmc_ctx *c, double ell, uint64_t seed, int32_t trial_sweeps,
                          ecmc_tuning *out) {
  if (!c || !out) return fail(ECMC_EINVAL, "NULL argument");
  if (!c->configured || c->opts.mode != ECMC_MODE_DOMAIN)
    return fail(ECMC_EINVAL, "autotune needs a context configured in the domain mode");
  if (trial_sweeps < 1 || !(ell > 0.0) || !isfinite(ell))
    return fail(ECMC_EINVAL, "need trial_sweeps >= 1 and a finite ell > 0");
  const ecmc_opts base = c->opts;
  const double sig = c->sigma;
  const double w = base.joint > 0 ? base.joint : c->b_max;
  const double halo_te = (c->b_max > sig ? c->b_max : sig) * (1.0 + 1e-6);
  // state on entry, restored before every trial and on return
  struct Saved {
    double *r = nullptr;
    int32_t *img = nullptr;
    ~Saved() {
      cudaFree(r);
      cudaFree(img);
    }
  } sv;
  CU(dalloc(&sv.r, 3 * c->n));
  CU(dalloc(&sv.img, 3 * c->n));
  unsigned long long cnt0[CNT_N];
  double sums0[SUM_N];
  CU(cudaMemcpyAsync(sv.r, c->d_r, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(sv.img, c->d_img, sizeof(int32_t) * 3 * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(cnt0, c->d_cnt, sizeof(cnt0), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(sums0, c->d_sums, sizeof(sums0), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  const int64_t sw0 = c->sweeps_done, ec0 = c->ecs_done;
  const double ds0 = c->device_seconds, es0 = c->ec_seconds;
  auto restore = [&]() -> ecmc_status {
    CU(cudaMemcpyAsync(c->d_r, sv.r, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_img, sv.img, sizeof(int32_t) * 3 * c->n, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_cnt, cnt0, sizeof(cnt0), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_sums, sums0, sizeof(sums0), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->sweeps_done = sw0;
    c->ecs_done = ec0;
    c->device_seconds = ds0;
    c->ec_seconds = es0;
    CU(mark_counters(c));  // the trials are no run to calibrate swaps on
    CU(cudaStreamSynchronize(c->stream));
    return ECMC_OK;
  };
  // the staging axes apply to the block-lockstep kernel only; elsewhere a
  // point off their defaults is not admissible (never timed)
  auto lock_point = [&](const TunePoint &pt) {
    return base.mode == ECMC_MODE_DOMAIN && base.precision == ECMC_PREC_FP32F && base.schedule == 0 &&
           base.k_spring == 0.0 && (pt.lanes == 4 || pt.lanes == 8 || pt.lanes == 16);
  };
  auto point_opts = [&](const TunePoint &pt) {
    ecmc_opts o = base;
    o.lanes = pt.lanes;
    o.cell_side = pt.cell_side * sig;
    o.ecs_per_tile = pt.ecs;
    o.stage_cap = 0;
    o.block_tiles = lock_point(pt) ? pt.warps * 32 / pt.lanes : 0;
    o.tight_factor = pt.tight;
    for (int a = 0; a < 3; ++a) {
      int D = (int)floor(c->L[a] / (pt.tile_side * sig));
      if (D < 3) D = 3;
      while (D < 1024 && !(c->L[a] / D - w + 2.0 * halo_te < 0.5 * c->L[a])) ++D;
      o.tiles[a] = D;
    }
    return o;
  };
  auto counts = [&](unsigned long long *h) -> ecmc_status {
    CU(cudaMemcpyAsync(h, c->d_cnt, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return ECMC_OK;
  };
  auto trial = [&](const TunePoint &pt, TuneScore *sc) -> ecmc_status {
    if (!lock_point(pt) && (pt.warps != 1 || pt.tight != 1.08)) return ECMC_EINVAL;
    ecmc_opts o = point_opts(pt);
    o.record = 0;
    ecmc_status st = ecmc_configure(c, &o);
    if (st != ECMC_OK) return st;
    if ((st = restore()) != ECMC_OK) return st;
    st = ecmc_run(c, ell, 0, seed, 1);
    if (st == ECMC_ECAPACITY) return ECMC_EINVAL;  // staging too small here: not admissible
    if (st != ECMC_OK) return st;
    unsigned long long h0[CNT_N], h1[CNT_N];
    if ((st = counts(h0)) != ECMC_OK) return st;
    const double t0 = c->device_seconds;
    st = ecmc_run(c, ell, 0, seed, trial_sweeps);
    if (st == ECMC_ECAPACITY) return ECMC_EINVAL;
    if (st != ECMC_OK) return st;
    if ((st = counts(h1)) != ECMC_OK) return st;
    const double dt = c->device_seconds - t0;
    if (!(dt > 0.0)) return ECMC_EINVAL;
    sc->ecs_per_s = (double)(h1[CNT_ECS] - h0[CNT_ECS]) / dt;
    sc->events_per_s = (double)(h1[CNT_EVENTS] - h0[CNT_EVENTS]) / dt;
    return ECMC_OK;
  };
  TunePoint start{c->lanes, c->T[0] / sig * (1.0 - 1e-9),
                  base.cell_side > 0 ? base.cell_side / sig : 1.05, c->ecs_per_tile, 1, 1.08};
  if (base.block_tiles > 0 && (c->lanes == 4 || c->lanes == 8 || c->lanes == 16))
    start.warps = base.block_tiles * c->lanes / 32;
  if (base.tight_factor > 0.0) start.tight = base.tight_factor;
  TunePoint best{};
  TuneScore best_s{};
  int n = 0;
  ecmc_status st = tune_search(start, trial, &best, &best_s, &n);
  if (st != ECMC_OK) {
    const std::string why = g_err;
    ecmc_configure(c, &base);
    restore();
    return fail(st, "autotune: %s", st == ECMC_EINVAL ? "no admissible setting" : why.c_str());
  }
  const ecmc_opts o = point_opts(best);
  if ((st = ecmc_configure(c, &o)) != ECMC_OK) return st;
  if ((st = restore()) != ECMC_OK) return st;
  out->lanes = best.lanes;
  out->tile_side = best.tile_side;
  out->cell_side = best.cell_side;
  out->ecs_per_tile = best.ecs;
  out->block_tiles = o.block_tiles;
  out->tight_factor = best.tight;
  for (int a = 0; a < 3; ++a) out->tiles[a] = o.tiles[a];
  out->ecs_per_s = best_s.ecs_per_s;
  out->events_per_s = best_s.events_per_s;
  out->n_trials = n;
  return ECMC_OK;
}

}  // extern "C"
