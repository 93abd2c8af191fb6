// Batched replicas (declared in ecmc.h): many independent melts advanced by
// one launch sequence per sweep — one domain assignment + cell list pass over
// all replicas' beads and one EC launch over all replicas' tiles — captured
// once in a CUDA graph and replayed; the sweep counter lives on the device.
// Replica r draws every random number with the Philox key (seed, r), so each
// replica evolves exactly as a single melt with that key would.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

using namespace ecmc;

namespace {
ecmc_status bfail(ecmc_status s, const std::string &msg) {
  set_last_error(msg.c_str());
  return s;
}
#define BCU(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return bfail(e_ == cudaErrorMemoryAllocation ? ECMC_ENOMEM : ECMC_ECUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

template <class T>
cudaError_t balloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (alloc_refused(sizeof(T) * count)) return cudaErrorMemoryAllocation;
  return cudaMalloc((void **)p, sizeof(T) * count);
}
}  // namespace

struct ecmc_batch {
  int32_t R = 0;
  std::vector<ecmc_replica_spec> specs;
  std::vector<RepParams> reps;
  int64_t n_total = 0, ncell_total = 0, units_total = 0;
  double sigma = 1.0, b_max = 1.2;
  uint64_t seed_lattice = 0;
  ecmc_opts opts{};
  bool configured = false;
  double s_cap = 0.25, halo_hs = 0, halo_te = 0;
  int32_t stage_cap = 0, m_cap = 0, ncl_max = 0, lanes = 8, ecs_per_tile = 1;
  int64_t event_cap = 10000000;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double *d_r = nullptr;
  int32_t *d_img = nullptr, *d_rep_of = nullptr, *d_tag = nullptr, *d_cell = nullptr,
          *d_rank = nullptr, *d_count = nullptr, *d_start = nullptr, *d_bsum = nullptr,
          *d_cid = nullptr, *d_ctag = nullptr;
  double *d_cr = nullptr;
  float *d_crf = nullptr, *d_rf = nullptr;
  RepParams *d_reps = nullptr;
  unsigned long long *d_cnt = nullptr;
  double *d_sums = nullptr;
  int *d_status = nullptr;
  int32_t *d_unit_next = nullptr;
  int32_t *d_n_deferred = nullptr, *d_deferred = nullptr;
  int64_t deferred_cap = 0;
  int32_t stage_tight = 0, m_tight = 0;
  int64_t *d_sweep = nullptr;
  uint64_t *d_rdig = nullptr;
  double *d_rlift = nullptr;
  int64_t *d_rev = nullptr;
  int64_t rec_cap = 0, rec_n = 0;
  cudaGraphExec_t graph = nullptr;
  double graph_ell = -1.0;
  uint64_t graph_seed = 0;
  bool graph_rec = false;
  int64_t graph_rec_sweep0 = -1;
  int64_t sweeps_done = 0;
  double device_seconds = 0.0;
};

namespace {

void batch_free(ecmc_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void *ptrs[] = {b->d_r, b->d_img, b->d_rep_of, b->d_tag, b->d_cell, b->d_rank, b->d_count,
                  b->d_start, b->d_bsum, b->d_cid, b->d_ctag, b->d_cr, b->d_crf, b->d_rf, b->d_reps,
                  b->d_cnt,
                  b->d_sums, b->d_status, b->d_unit_next, b->d_n_deferred, b->d_deferred, b->d_sweep,
                  b->d_rdig, b->d_rlift,
                  b->d_rev};
  for (void *p : ptrs) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

ecmc_status batch_status(ecmc_batch *b) {
  int st = 0;
  BCU(cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  if (st == DEV_STUCK) return bfail(ECMC_ESTUCK, "an event chain exceeded the event cap");
  if (st == DEV_CAPACITY) return bfail(ECMC_ECAPACITY, "a tile exceeded the staging capacity");
  if (st == DEV_TILE) return bfail(ECMC_ECAPACITY, "a bonded partner was not staged with its tile");
  return ECMC_OK;
}

// one sweep of every replica: domain assignment + cell list, EC kernel,
// sweep counter advance (all stream-ordered, so it can be captured)
cudaError_t batch_sweep(ecmc_batch *b, const ECParams &P, uint64_t seed) {
  CellBatch C{};
  C.n = b->n_total;
  C.r = b->d_r;
  C.rep_of = b->d_rep_of;
  C.reps = b->d_reps;
  C.seed = seed;
  C.sweep_dev = b->d_sweep;
  C.tag = b->d_tag;
  C.cell = b->d_cell;
  C.rank = b->d_rank;
  C.count = b->d_count;
  C.start = b->d_start;
  C.block_sums = b->d_bsum;
  C.cr = b->d_cr;
  C.crf = b->d_crf;
  C.rf = b->d_rf;
  C.cid = b->d_cid;
  C.ctag = b->d_ctag;
  cudaError_t e = launch_cells_batch(C, b->ncell_total, b->stream);
  if (e != cudaSuccess) return e;
  const bool lock = b->opts.precision == ECMC_PREC_FP32F && b->opts.schedule == 0 &&
                    (b->lanes == 4 || b->lanes == 8 || b->lanes == 16);
  e = lock ? launch_ec_lock_batch(P, b->lanes, b->stream)
           : launch_ec_batch(P, b->lanes, b->opts.precision == ECMC_PREC_FP32F, b->stream);
  if (e != cudaSuccess) return e;
  return launch_sweep_advance(b->d_sweep, b->stream);
}

ECParams batch_params(ecmc_batch *b, uint64_t seed, double ell) {
  ECParams P{};
  P.n = b->n_total;
  P.sigma = b->sigma;
  P.sig2 = b->sigma * b->sigma;
  P.b2 = b->b_max * b->b_max;
  P.s_cap = b->s_cap;
  P.s_cap_f = round_up_f32(b->s_cap);
  P.domain = 1;
  P.halo_hs = b->halo_hs;
  P.halo_te = b->halo_te;
  P.seed = seed;
  P.ell = ell;
  P.event_cap = b->event_cap;
  P.p_swap = b->opts.p_swap;
  P.swap_mode = b->opts.p_swap >= 1.0 ? 1 : (b->opts.p_swap > 0.0 ? 2 : 0);
  P.swap_thr = P.swap_mode == 2 ? (uint64_t)ceil(b->opts.p_swap * 9007199254740992.0) : 0;
  P.dir_mode = b->opts.dir_mode;
  P.stage_cap = b->stage_cap;
  P.m_cap = b->m_cap;
  P.n_units = (int32_t)b->units_total;
  P.ecs_per_tile = b->ecs_per_tile;
  double Lm = 0.0;
  for (const RepParams &R : b->reps)
    for (int a = 0; a < 3; ++a) Lm = R.L[a] > Lm ? R.L[a] : Lm;
  const double err = (3.0 * Lm + 64.0 * b->sigma) / 16777216.0;
  const double ev = 35.0 * err > 2e-4 * b->sigma ? 35.0 * err : 2e-4 * b->sigma;
  const double ed = 180.0 * err * b->sigma > 1e-3 * b->sigma * b->sigma ? 180.0 * err * b->sigma
                                                                       : 1e-3 * b->sigma * b->sigma;
  P.eps_v = (float)ev;
  P.eps_d = (float)ed;
  P.eps_x = (float)ev;
  P.r = b->d_r;
  P.img = b->d_img;
  P.cr = b->d_cr;
  P.crf = b->d_crf;
  P.rf = b->d_rf;
  P.cid = b->d_cid;
  P.ctag = b->d_ctag;
  P.cstart = b->d_start;
  P.counters = b->d_cnt;
  P.sums = b->d_sums;
  P.status = b->d_status;
  P.reps = b->d_reps;
  P.n_reps = b->R;
  P.ncl_max = b->ncl_max;
  P.sweep_dev = b->d_sweep;
  P.block_tiles = b->opts.block_tiles;
  P.rq_per_tile = b->opts.request_cap > 0 ? b->opts.request_cap : 6;
  P.unit_next = b->d_unit_next;
  P.stage_tight = b->stage_tight;
  P.m_tight = b->m_tight;
  P.deferred = b->d_deferred;
  P.n_deferred = b->d_n_deferred;
  return P;
}

}  // namespace

extern "C" {

ecmc_status ecmc_batch_create(const ecmc_replica_spec *specs, int32_t n, double jitter,
                              uint64_t seed, ecmc_batch **out) {
  if (!specs || !out || n < 1) return bfail(ECMC_EINVAL, "need at least one replica spec");
  *out = nullptr;
  const double sigma = specs[0].sigma, b_max = specs[0].b_max;
  if (!(sigma > 0.0) || !(b_max >= sigma)) return bfail(ECMC_EINVAL, "need 0 < sigma <= b_max");
  int64_t n_total = 0;
  for (int32_t r = 0; r < n; ++r) {
    const ecmc_replica_spec &sp = specs[r];
    if (sp.sigma != sigma || sp.b_max != b_max)
      return bfail(ECMC_EINVAL, "all replicas need the same sigma and b_max");
    if (sp.dims[0] < 1 || sp.dims[1] < 1 || sp.dims[2] < 1 || sp.N < 1)
      return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": bad dims or N");
    const int64_t nb = (int64_t)sp.dims[0] * sp.dims[1] * sp.dims[2];
    if (nb % sp.N) return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": N must divide the sites");
    if (!(sp.spacing >= sigma) || (sp.N > 1 && !(sp.spacing <= b_max)))
      return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": need sigma <= spacing <= b_max");
    if (jitter < 0.0 || (jitter > 0.0 && !(2.0 * jitter < sp.spacing - sigma)))
      return bfail(ECMC_EINVAL, "jitter must be in [0, (spacing - sigma)/2)");
    n_total += nb;
  }
  if (n_total >= (1ll << 31)) return bfail(ECMC_EINVAL, "at most 2^31 beads in a batch");
  ecmc_batch *b = new ecmc_batch();
  b->R = n;
  b->specs.assign(specs, specs + n);
  b->sigma = sigma;
  b->b_max = b_max;
  b->seed_lattice = seed;
  b->n_total = n_total;
  b->reps.resize(n);
  std::vector<int32_t> rep_of(n_total);
  int64_t off = 0;
  for (int32_t r = 0; r < n; ++r) {
    RepParams &R = b->reps[r];
    memset(&R, 0, sizeof(R));
    const ecmc_replica_spec &sp = specs[r];
    for (int a = 0; a < 3; ++a) {
      R.L[a] = sp.dims[a] * sp.spacing;
      R.half[a] = 0.5 * R.L[a];
    }
    R.N = sp.N;
    R.bead_off = off;
    R.n_beads = (int64_t)sp.dims[0] * sp.dims[1] * sp.dims[2];
    R.replica = (uint64_t)r;
    for (int64_t i = 0; i < R.n_beads; ++i) rep_of[off + i] = r;
    off += R.n_beads;
  }
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = balloc(&b->d_r, 3 * n_total);
  if (e == cudaSuccess) e = balloc(&b->d_img, 3 * n_total);
  if (e == cudaSuccess) e = balloc(&b->d_rep_of, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_tag, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_cell, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_rank, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_cr, 3 * n_total);
  if (e == cudaSuccess) e = balloc(&b->d_crf, 3 * n_total);
  if (e == cudaSuccess) e = balloc(&b->d_rf, 3 * n_total);
  if (e == cudaSuccess) e = balloc(&b->d_cid, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_ctag, n_total);
  if (e == cudaSuccess) e = balloc(&b->d_reps, n);
  if (e == cudaSuccess) e = balloc(&b->d_cnt, CNT_N);
  if (e == cudaSuccess) e = balloc(&b->d_sums, SUM_N);
  if (e == cudaSuccess) e = balloc(&b->d_status, 1);
  if (e == cudaSuccess) e = balloc(&b->d_unit_next, 1);
  if (e == cudaSuccess) e = balloc(&b->d_n_deferred, 1);
  if (e == cudaSuccess) e = balloc(&b->d_sweep, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_img, 0, sizeof(int32_t) * 3 * n_total, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cnt, 0, sizeof(unsigned long long) * CNT_N, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_sums, 0, sizeof(double) * SUM_N, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_rep_of, rep_of.data(), sizeof(int32_t) * n_total,
                        cudaMemcpyHostToDevice, b->stream);
  for (int32_t r = 0; r < n && e == cudaSuccess; ++r)
    e = launch_lattice(specs[r].dims, specs[r].spacing, jitter, seed, (uint64_t)r,
                       b->d_r + 3 * b->reps[r].bead_off, b->reps[r].n_beads, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    batch_free(b);
    return bfail(e == cudaErrorMemoryAllocation ? ECMC_ENOMEM : ECMC_ECUDA,
                 std::string("batch create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return ECMC_OK;
}

void ecmc_batch_destroy(ecmc_batch *b) { batch_free(b); }

ecmc_status ecmc_batch_configure(ecmc_batch *b, const ecmc_opts *o) {
  if (!b || !o) return bfail(ECMC_EINVAL, "NULL argument");
  ecmc_opts p = *o;
  if (p.mode != ECMC_MODE_DOMAIN) return bfail(ECMC_EINVAL, "a batch runs in the domain mode");
  if (p.dir_mode != ECMC_DIR_CART3 && p.dir_mode != ECMC_DIR_ISO) return bfail(ECMC_EINVAL, "bad dir_mode");
  if (p.precision != ECMC_PREC_FP64 && p.precision != ECMC_PREC_FP32F)
    return bfail(ECMC_EINVAL, "bad precision");
  const int lanes = p.lanes ? p.lanes : 8;
  if (lanes != 32 && lanes != 16 && lanes != 8 && lanes != 4)
    return bfail(ECMC_EINVAL, "batch lanes must be 4, 8, 16 or 32");
  if (!(p.p_swap >= 0.0)) return bfail(ECMC_EINVAL, "p_swap must be >= 0");
  if (p.k_spring != 0.0) return bfail(ECMC_EINVAL, "the batch runs hard tethers (k_spring must be 0)");
  const double sig = b->sigma;
  const double s_cap = p.s_cap > 0 ? p.s_cap : 0.25 * sig;
  const double w = p.joint > 0 ? p.joint : b->b_max;
  if (!(w >= b->b_max)) return bfail(ECMC_EINVAL, "joint width must be >= b_max");
  const double side = p.cell_side > 0 ? p.cell_side : 1.05 * sig;
  if (!(side >= sig)) return bfail(ECMC_EINVAL, "cell side must be >= sigma");
  const double tside = p.tile_side > 0 ? p.tile_side : 4.2 * sig;
  const double halo_hs = sig * (1.0 + 1e-6);
  const double halo_te = (b->b_max > sig ? b->b_max : sig) * (1.0 + 1e-6);
  const double hg = halo_te + 1e-3 * sig;
  const double reach = s_cap + sig + 0.01 * sig;
  const double bm = b->b_max * (1.0 + 1e-6);
  const double side_min = (reach > bm ? reach : bm) + 2e-3 * sig;
  const double margin = p.precision == ECMC_PREC_FP32F ? 0.01 * sig : 0.0;
  int64_t cell_off = 0, unit_off = 0;
  int32_t stage = 0, mcap = 0, nclm = 0, stage_t = 0, m_t = 0;
  std::vector<RepParams> reps = b->reps;
  for (int32_t r = 0; r < b->R; ++r) {
    RepParams &R = reps[r];
    const double rho = (double)R.n_beads / (R.L[0] * R.L[1] * R.L[2]);
    int64_t ncl = 1, nce = 1, nt = 1;
    for (int a = 0; a < 3; ++a) {
      if (!(s_cap + sig + margin < R.half[a]))
        return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": need s_cap + sigma < L/2");
      int D = p.tiles[a] > 0 ? p.tiles[a] : (int)floor(R.L[a] / tside);
      if (D < 3) D = 3;
      // the tile plus its halo must stay below half the box
      while (D < 1024 && !(R.L[a] / D - w + 2.0 * halo_te < R.half[a])) ++D;
      const double T = R.L[a] / D, W = T - w;
      if (!(W > 0.0))
        return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": tile narrower than the joint");
      if (p.precision == ECMC_PREC_FP32F && !(W + 2.0 * halo_te <= 64.0 * sig))
        return bfail(ECMC_EINVAL, "FP32 screen needs tiles of at most 64 sigma");
      R.D[a] = D;
      R.T[a] = T;
      R.W[a] = W;
      int k = (int)floor(R.L[a] / side);
      if (k < 3) return bfail(ECMC_EINVAL, "replica " + std::to_string(r) + ": box too small");
      R.nc[a] = k;
      R.cs[a] = R.L[a] / k;
      const double E = W + 2.0 * hg;
      int g = (int)floor(E / side_min);
      if (g < 1) g = 1;
      R.lg[a] = g;
      R.linv[a] = (float)(g / E);
      ncl *= g;
      nce *= k;
      nt *= D;
    }
    R.lorg = (float)(-hg);
    R.cell_off = cell_off;
    R.unit_off = unit_off;
    cell_off += nce;
    unit_off += nt;
    const double E[3] = {R.W[0] + 2.0 * halo_te, R.W[1] + 2.0 * halo_te, R.W[2] + 2.0 * halo_te};
    const int32_t st = stage_bound(E, rho);
    const int32_t mc = stage_bound(R.W, rho);
    stage = st > stage ? st : stage;
    mcap = mc > mcap ? mc : mcap;
    int32_t st_t = 0, mc_t = 0;
    tight_caps(E, R.W, rho, st, mc, &st_t, &mc_t, p.tight_factor > 0 ? p.tight_factor : 1.08);
    stage_t = st_t > stage_t ? st_t : stage_t;
    m_t = mc_t > m_t ? mc_t : m_t;
    nclm = (int32_t)ncl > nclm ? (int32_t)ncl : nclm;
  }
  if (p.stage_cap > 0) {
    stage = (p.stage_cap + 31) / 32 * 32;
    stage_t = m_t = 0;  // caller-fixed capacity: one pass
  }
  if (m_t > stage_t) m_t = stage_t;
  if (mcap > stage) mcap = stage;
  if (stage > 65534) return bfail(ECMC_EINVAL, "at most 65534 staged beads per tile");
  if (unit_off >= (1ll << 31)) return bfail(ECMC_EINVAL, "too many tiles");
  int dev = 0, smem_max = 0;
  BCU(cudaGetDevice(&dev));
  BCU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int M = p.precision == ECMC_PREC_FP32F ? mcap : stage;
  if (p.schedule != 0 && p.schedule != 1) return bfail(ECMC_EINVAL, "schedule must be 0 or 1");
  if (p.block_tiles < 0 || p.block_tiles > 32 || p.block_tiles * lanes > 128 ||
      (p.block_tiles > 0 && p.block_tiles % (32 / lanes)))
    return bfail(ECMC_EINVAL, "block_tiles must be a multiple of 32 / lanes, at most 32 and 128 / lanes");
  if (p.request_cap < 0 || p.request_cap > 6) return bfail(ECMC_EINVAL, "request_cap must be in [0, 6]");
  const bool lock = p.precision == ECMC_PREC_FP32F && p.schedule == 0 && lanes <= 16;
  const int bt = p.block_tiles > 0 ? p.block_tiles : 32 / lanes;
  const size_t need = lock ? lock_smem_bytes(stage, M, nclm, bt) : ec_smem_bytes(stage, M, nclm, 32 / lanes);
  if ((int64_t)need > smem_max)
    return bfail(ECMC_EINVAL, "staging does not fit in shared memory");
  // (re)allocate the concatenated cell arrays
  if (cell_off != b->ncell_total) {
    cudaFree(b->d_count);
    cudaFree(b->d_start);
    cudaFree(b->d_bsum);
    b->d_count = b->d_start = b->d_bsum = nullptr;
    BCU(balloc(&b->d_count, cell_off));
    BCU(balloc(&b->d_start, cell_off + 1));
    BCU(balloc(&b->d_bsum, cells_scratch_ints(cell_off)));
    b->ncell_total = cell_off;
  }
  b->reps = reps;
  BCU(cudaMemcpyAsync(b->d_reps, b->reps.data(), sizeof(RepParams) * b->R, cudaMemcpyHostToDevice,
                      b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  b->opts = p;
  b->opts.lanes = lanes;
  b->opts.tile_side = tside;
  b->s_cap = s_cap;
  b->halo_hs = halo_hs;
  b->halo_te = halo_te;
  b->stage_cap = stage;
  b->m_cap = mcap;
  b->stage_tight = stage_t;
  b->m_tight = m_t;
  if (unit_off > b->deferred_cap) {
    cudaFree(b->d_deferred);
    b->d_deferred = nullptr;
    b->deferred_cap = 0;
    BCU(balloc(&b->d_deferred, unit_off));
    b->deferred_cap = unit_off;
  }
  b->ncl_max = nclm;
  b->lanes = lanes;
  b->ecs_per_tile = p.ecs_per_tile > 0 ? p.ecs_per_tile : 1;
  b->event_cap = p.event_cap > 0 ? p.event_cap : 10000000;
  b->units_total = unit_off;
  b->configured = true;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return ECMC_OK;
}

ecmc_status ecmc_batch_run(ecmc_batch *b, double ell, uint64_t seed, int64_t n_sweeps,
                           int32_t use_graph) {
  if (!b) return bfail(ECMC_EINVAL, "batch is NULL");
  if (!b->configured) return bfail(ECMC_EINVAL, "call ecmc_batch_configure first");
  if (!(ell >= 0.0) || !isfinite(ell) || n_sweeps < 0) return bfail(ECMC_EINVAL, "bad ell or n_sweeps");
  const bool rec = b->opts.record != 0;
  ECParams P = batch_params(b, seed, ell);
  if (rec) {
    const int64_t units = n_sweeps * b->units_total * b->ecs_per_tile;
    if (units > b->rec_cap) {
      cudaFree(b->d_rdig);
      cudaFree(b->d_rlift);
      cudaFree(b->d_rev);
      b->d_rdig = nullptr;
      b->d_rlift = nullptr;
      b->d_rev = nullptr;
      b->rec_cap = 0;
      BCU(balloc(&b->d_rdig, units));
      BCU(balloc(&b->d_rlift, units));
      BCU(balloc(&b->d_rev, units));
      b->rec_cap = units;
    }
    BCU(cudaMemsetAsync(b->d_rdig, 0, sizeof(uint64_t) * (units ? units : 1), b->stream));
    b->rec_n = units;
    P.rec_digest = b->d_rdig;
    P.rec_lift = b->d_rlift;
    P.rec_events = b->d_rev;
    P.rec_cap = b->rec_cap;
    P.rec_sweep0 = b->sweeps_done;
  }
  BCU(cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
  BCU(cudaMemcpyAsync(b->d_sweep, &b->sweeps_done, sizeof(int64_t), cudaMemcpyHostToDevice,
                      b->stream));
  BCU(cudaEventRecord(b->ev0, b->stream));
  if (use_graph && n_sweeps > 0) {
    // records bake their buffers and sweep base into the graph: recapture
    const bool fresh = rec || !b->graph || b->graph_ell != ell || b->graph_seed != seed ||
                       b->graph_rec != rec;
    int64_t done = 0;
    if (fresh) {
      if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
      }
      // first sweep uncaptured: kernel attributes and block sizes are
      // settled outside the capture
      BCU(batch_sweep(b, P, seed));
      done = 1;
      cudaGraph_t g = nullptr;
      BCU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
      cudaError_t e = batch_sweep(b, P, seed);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(ECMC_ECUDA, std::string("graph capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return bfail(ECMC_ECUDA, std::string("graph: ") + cudaGetErrorString(e));
      b->graph_ell = ell;
      b->graph_seed = seed;
      b->graph_rec = rec;
      b->graph_rec_sweep0 = b->sweeps_done;
    }
    for (int64_t s = done; s < n_sweeps; ++s) BCU(cudaGraphLaunch(b->graph, b->stream));
  } else {
    for (int64_t s = 0; s < n_sweeps; ++s) BCU(batch_sweep(b, P, seed));
  }
  BCU(cudaEventRecord(b->ev1, b->stream));
  ecmc_status st = batch_status(b);
  float ms = 0.f;
  BCU(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
  b->device_seconds += 1e-3 * ms;
  b->sweeps_done += n_sweeps;
  return st;
}

ecmc_status ecmc_batch_get_positions(ecmc_batch *b, int32_t replica, double *xyz, int32_t *img) {
  if (!b || !xyz || replica < 0 || replica >= b->R) return bfail(ECMC_EINVAL, "bad argument");
  const RepParams &R = b->reps[replica];
  BCU(cudaMemcpyAsync(xyz, b->d_r + 3 * R.bead_off, sizeof(double) * 3 * R.n_beads,
                      cudaMemcpyDeviceToHost, b->stream));
  if (img)
    BCU(cudaMemcpyAsync(img, b->d_img + 3 * R.bead_off, sizeof(int32_t) * 3 * R.n_beads,
                        cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  return ECMC_OK;
}

ecmc_status ecmc_batch_info(ecmc_batch *b, int32_t replica, int32_t tiles[3], int64_t *unit_off,
                            int64_t *n_beads) {
  if (!b || replica < 0 || replica >= b->R) return bfail(ECMC_EINVAL, "bad argument");
  const RepParams &R = b->reps[replica];
  if (tiles)
    for (int a = 0; a < 3; ++a) tiles[a] = R.D[a];
  if (unit_off) *unit_off = R.unit_off;
  if (n_beads) *n_beads = R.n_beads;
  return ECMC_OK;
}

ecmc_status ecmc_batch_stats(ecmc_batch *b, int64_t *events_total, int64_t *ecs,
                             double *device_seconds) {
  if (!b) return bfail(ECMC_EINVAL, "batch is NULL");
  unsigned long long h[CNT_N];
  BCU(cudaMemcpyAsync(h, b->d_cnt, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  if (events_total) *events_total = (int64_t)h[CNT_EVENTS];
  if (ecs) *ecs = (int64_t)h[CNT_ECS];
  if (device_seconds) *device_seconds = b->device_seconds;
  return ECMC_OK;
}

ecmc_status ecmc_batch_records(ecmc_batch *b, uint64_t *digest, double *lift, int64_t *events,
                               int64_t *n) {
  if (!b || !n) return bfail(ECMC_EINVAL, "NULL argument");
  if (!b->d_rdig) {
    *n = 0;
    return ECMC_OK;
  }
  const int64_t cnt = b->rec_n < *n ? b->rec_n : *n;
  if (digest) BCU(cudaMemcpyAsync(digest, b->d_rdig, sizeof(uint64_t) * cnt, cudaMemcpyDeviceToHost, b->stream));
  if (lift) BCU(cudaMemcpyAsync(lift, b->d_rlift, sizeof(double) * cnt, cudaMemcpyDeviceToHost, b->stream));
  if (events) BCU(cudaMemcpyAsync(events, b->d_rev, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  *n = cnt;
  return ECMC_OK;
}

ecmc_status ecmc_batch_autotune(ecmc_batch *b, double ell, uint64_t seed, int32_t trial_sweeps,
                                ecmc_tuning *out) {
  if (!b || !out) return bfail(ECMC_EINVAL, "NULL argument");
  if (!b->configured) return bfail(ECMC_EINVAL, "call ecmc_batch_configure first");
  if (trial_sweeps < 1 || !(ell > 0.0) || !isfinite(ell))
    return bfail(ECMC_EINVAL, "need trial_sweeps >= 1 and a finite ell > 0");
  const ecmc_opts base = b->opts;
  const double sig = b->sigma;
  struct Saved {
    double *r = nullptr;
    int32_t *img = nullptr;
    ~Saved() {
      cudaFree(r);
      cudaFree(img);
    }
  } sv;
  const int64_t n3 = 3 * b->n_total;
  BCU(balloc(&sv.r, n3));
  BCU(balloc(&sv.img, n3));
  unsigned long long cnt0[CNT_N];
  double sums0[SUM_N];
  BCU(cudaMemcpyAsync(sv.r, b->d_r, sizeof(double) * n3, cudaMemcpyDeviceToDevice, b->stream));
  BCU(cudaMemcpyAsync(sv.img, b->d_img, sizeof(int32_t) * n3, cudaMemcpyDeviceToDevice, b->stream));
  BCU(cudaMemcpyAsync(cnt0, b->d_cnt, sizeof(cnt0), cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaMemcpyAsync(sums0, b->d_sums, sizeof(sums0), cudaMemcpyDeviceToHost, b->stream));
  BCU(cudaStreamSynchronize(b->stream));
  const int64_t sw0 = b->sweeps_done;
  const double ds0 = b->device_seconds;
  auto restore = [&]() -> ecmc_status {
    BCU(cudaMemcpyAsync(b->d_r, sv.r, sizeof(double) * n3, cudaMemcpyDeviceToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_img, sv.img, sizeof(int32_t) * n3, cudaMemcpyDeviceToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_cnt, cnt0, sizeof(cnt0), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaMemcpyAsync(b->d_sums, sums0, sizeof(sums0), cudaMemcpyHostToDevice, b->stream));
    BCU(cudaStreamSynchronize(b->stream));
    b->sweeps_done = sw0;
    b->device_seconds = ds0;
    return ECMC_OK;
  };
  // the staging axes apply to the block-lockstep kernel only
  auto lock_point = [&](const TunePoint &pt) {
    return base.precision == ECMC_PREC_FP32F && base.schedule == 0 &&
           (pt.lanes == 4 || pt.lanes == 8 || pt.lanes == 16);
  };
  auto point_opts = [&](const TunePoint &pt) {
    ecmc_opts o = base;
    o.lanes = pt.lanes;
    o.tile_side = pt.tile_side * sig;
    o.tiles[0] = o.tiles[1] = o.tiles[2] = 0;
    o.cell_side = pt.cell_side * sig;
    o.ecs_per_tile = pt.ecs;
    o.stage_cap = 0;
    o.block_tiles = lock_point(pt) ? pt.warps * 32 / pt.lanes : 0;
    o.tight_factor = pt.tight;
    return o;
  };
  auto trial = [&](const TunePoint &pt, TuneScore *sc) -> ecmc_status {
    if (!lock_point(pt) && (pt.warps != 1 || pt.tight != 1.08)) return ECMC_EINVAL;
    ecmc_opts o = point_opts(pt);
    o.record = 0;
    ecmc_status st = ecmc_batch_configure(b, &o);
    if (st != ECMC_OK) return st;
    if ((st = restore()) != ECMC_OK) return st;
    // the first call settles block sizes and captures the sweep graph
    st = ecmc_batch_run(b, ell, seed, 1, 1);
    if (st == ECMC_ECAPACITY) return ECMC_EINVAL;
    if (st != ECMC_OK) return st;
    int64_t e0 = 0, c0 = 0, e1 = 0, c1 = 0;
    double t0 = 0, t1 = 0;
    if ((st = ecmc_batch_stats(b, &e0, &c0, &t0)) != ECMC_OK) return st;
    st = ecmc_batch_run(b, ell, seed, trial_sweeps, 1);
    if (st == ECMC_ECAPACITY) return ECMC_EINVAL;
    if (st != ECMC_OK) return st;
    if ((st = ecmc_batch_stats(b, &e1, &c1, &t1)) != ECMC_OK) return st;
    const double dt = t1 - t0;
    if (!(dt > 0.0)) return ECMC_EINVAL;
    sc->ecs_per_s = (double)(c1 - c0) / dt;
    sc->events_per_s = (double)(e1 - e0) / dt;
    return ECMC_OK;
  };
  TunePoint start{b->lanes, base.tile_side / sig, base.cell_side > 0 ? base.cell_side / sig : 1.05,
                  b->ecs_per_tile, 1, 1.08};
  if (base.block_tiles > 0 && (b->lanes == 4 || b->lanes == 8 || b->lanes == 16))
    start.warps = base.block_tiles * b->lanes / 32;
  if (base.tight_factor > 0.0) start.tight = base.tight_factor;
  TunePoint best{};
  TuneScore best_s{};
  int n = 0;
  ecmc_status st = tune_search(start, trial, &best, &best_s, &n);
  if (st != ECMC_OK) {
    ecmc_batch_configure(b, &base);
    restore();
    return bfail(st, st == ECMC_EINVAL ? "autotune: no admissible setting" : "autotune failed");
  }
  const ecmc_opts o = point_opts(best);
  if ((st = ecmc_batch_configure(b, &o)) != ECMC_OK) return st;
  if ((st = restore()) != ECMC_OK) return st;
  out->lanes = best.lanes;
  out->tile_side = best.tile_side;
  out->cell_side = best.cell_side;
  out->ecs_per_tile = best.ecs;
  out->block_tiles = o.block_tiles;
  out->tight_factor = best.tight;
  out->tiles[0] = out->tiles[1] = out->tiles[2] = 0;
  out->ecs_per_s = best_s.ecs_per_s;
  out->events_per_s = best_s.events_per_s;
  out->n_trials = n;
  return ECMC_OK;
}

}  // extern "C"
