// ecmc_cells_static: the domain assignment and cell list of one sweep for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option, e.g.
// inside a host callback or a framework whose allocator owns all device
// memory, or a real-time loop that must not hit the driver's allocator.
// Such callers pass their own device buffers for the inputs and outputs;
// the temporary arrays of the counting sort (per-bead ranks, per-cell
// counts, scan block sums) live in one file-scope __device__ array instead,
// which every GPU that loads this library holds until the process exits.
//
// The computation is the same as the library's per-sweep domain assignment:
// shift o from Philox (tag 2, counter (2, sweep, 0, 0), key (seed, 0)), tile
// of every bead or -1 for the joint, and beads binned into the cell grid
// nc_a = floor(L_a / cell_side) (order inside a cell not fixed).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

constexpr int64_t STATIC_MAX_BEADS = 1 << 20;
constexpr int64_t STATIC_MAX_CELLS = 1 << 20;
constexpr int ST_BLOCK = 1024;
constexpr int ST_ITEMS = 4;
constexpr int64_t ST_TILE = ST_BLOCK * ST_ITEMS;
constexpr int64_t ST_MAX_TILES = (STATIC_MAX_CELLS + ST_TILE - 1) / ST_TILE;
// [0, MAX_BEADS): rank of each bead in its cell; [MAX_BEADS, +MAX_CELLS):
// per-cell counts; then the scan block sums
constexpr int64_t SCRATCH_INTS = STATIC_MAX_BEADS + STATIC_MAX_CELLS + ST_MAX_TILES + 1;

static __device__ __align__(256) int32_t g_scratch[SCRATCH_INTS];

struct StaticParams {
  const double *r;
  int64_t n;
  double L[3];
  int32_t nc[3];
  double cs[3];
  int32_t D[3];
  double T[3], W[3];
  uint64_t seed;
  int64_t sweep;
  int32_t *tags;
  int32_t *start;
  int32_t *ids;
  int32_t *rank;
  int32_t *count;
  int32_t *bsum;
};

__device__ __forceinline__ int cell_of(const StaticParams &S, double r0, double r1, double r2) {
  const double rr[3] = {r0, r1, r2};
  int c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int t = (int)(rr[a] / S.cs[a]);
    if (t >= S.nc[a]) t = S.nc[a] - 1;
    if (t < 0) t = 0;
    c[a] = t;
  }
  return (c[2] * S.nc[1] + c[1]) * S.nc[0] + c[0];
}

__global__ void ks_tag_count(const StaticParams S) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.n) return;
  const double rr[3] = {S.r[3 * b], S.r[3 * b + 1], S.r[3 * b + 2]};
  const u64x4 w = philox(TAG_SHIFT, (uint64_t)S.sweep, 0, 0, S.seed, 0);
  int k[3];
  bool in = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double o = unit53(w.v[a]) * S.T[a];
    double u = rr[a] - o;
    if (u < 0.0) u = u + S.L[a];
    if (u >= S.L[a]) u = u - S.L[a];
    int t = (int)(u / S.T[a]);
    if (t > S.D[a] - 1) t = S.D[a] - 1;
    const double loc = u - (double)t * S.T[a];
    in = in && (loc < S.W[a]);
    k[a] = t;
  }
  S.tags[b] = in ? (k[2] * S.D[1] + k[1]) * S.D[0] + k[0] : -1;
  S.rank[b] = atomicAdd(&S.count[cell_of(S, rr[0], rr[1], rr[2])], 1);
}

__device__ int st_block_scan(int (&v)[ST_ITEMS], int *sh) {
  int local = 0;
#pragma unroll
  for (int i = 0; i < ST_ITEMS; ++i) {
    const int t = v[i];
    v[i] = local;
    local += t;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = local;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int w = sh[lane];
    int wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const int base = sh[wid] + inc - local;
#pragma unroll
  for (int i = 0; i < ST_ITEMS; ++i) v[i] += base;
  const int total = sh[32];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(ST_BLOCK) ks_scan_tiles(const StaticParams S, int64_t ncell) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * ST_TILE + (int64_t)threadIdx.x * ST_ITEMS;
  int v[ST_ITEMS];
#pragma unroll
  for (int i = 0; i < ST_ITEMS; ++i) v[i] = (base + i < ncell) ? S.count[base + i] : 0;
  const int total = st_block_scan(v, sh);
#pragma unroll
  for (int i = 0; i < ST_ITEMS; ++i)
    if (base + i < ncell) S.start[base + i] = v[i];
  if (threadIdx.x == 0) S.bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(ST_BLOCK) ks_scan_sums(const StaticParams S, int64_t tiles,
                                                         int64_t ncell) {
  __shared__ int sh[33];
  int carry = 0;
  for (int64_t c0 = 0; c0 < tiles; c0 += ST_TILE) {
    const int64_t base = c0 + (int64_t)threadIdx.x * ST_ITEMS;
    int v[ST_ITEMS];
#pragma unroll
    for (int i = 0; i < ST_ITEMS; ++i) v[i] = (base + i < tiles) ? S.bsum[base + i] : 0;
    const int total = st_block_scan(v, sh);
#pragma unroll
    for (int i = 0; i < ST_ITEMS; ++i)
      if (base + i < tiles) S.bsum[base + i] = v[i] + carry;
    carry += total;
  }
  if (threadIdx.x == 0) S.start[ncell] = carry;
}

__global__ void ks_scan_add(const StaticParams S, int64_t ncell) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncell) S.start[i] += S.bsum[i / ST_TILE];
}

__global__ void ks_scatter(const StaticParams S) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= S.n) return;
  const int c = cell_of(S, S.r[3 * b], S.r[3 * b + 1], S.r[3 * b + 2]);
  S.ids[(int64_t)S.start[c] + S.rank[b]] = (int32_t)b;
}

// device address of g_scratch, looked up once per device and kept for the
// life of the process (a cudaDeviceReset of that device makes it stale; the
// header says so)
std::mutex g_mu;
int32_t *g_ptr[256] = {nullptr};

cudaError_t scratch_for_current_device(int32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = (int32_t *)p;
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ecmc

using namespace ecmc;

extern "C" ecmc_status ecmc_cells_static(const double *d_r, int64_t n, const double box[3],
                                         const int32_t tiles[3], double joint, double cell_side,
                                         uint64_t seed, int64_t sweep, int32_t *d_tags,
                                         int32_t *d_cell_start, int32_t *d_cell_ids,
                                         double shift_out[3], void *stream) {
  if (!d_r || !box || !tiles || !d_tags || !d_cell_start || !d_cell_ids) {
    set_last_error("ecmc_cells_static: NULL argument");
    return ECMC_EINVAL;
  }
  if (n < 1 || n > STATIC_MAX_BEADS) {
    set_last_error("ecmc_cells_static: n must be in [1, 1048576]");
    return ECMC_EINVAL;
  }
  if (!(cell_side > 0.0) || !(joint > 0.0)) {
    set_last_error("ecmc_cells_static: cell_side and joint must be > 0");
    return ECMC_EINVAL;
  }
  StaticParams S{};
  // every count is bounded while still in double, before any integer cast
  // or product: per axis at most STATIC_MAX_CELLS cells, the grid at most
  // STATIC_MAX_CELLS after every multiply, the tile count within int32
  int64_t ncell = 1, ntile = 1;
  for (int a = 0; a < 3; ++a) {
    if (!(box[a] > 0.0 && box[a] < INFINITY) || tiles[a] < 1) {
      set_last_error("ecmc_cells_static: box must be finite and > 0 and tiles >= 1");
      return ECMC_EINVAL;
    }
    const double kd = floor(box[a] / cell_side);
    if (!(kd >= 1.0)) {
      set_last_error("ecmc_cells_static: cell_side larger than the box");
      return ECMC_EINVAL;
    }
    if (!(kd <= (double)STATIC_MAX_CELLS)) {
      set_last_error("ecmc_cells_static: more than 1048576 cells");
      return ECMC_EINVAL;
    }
    const int k = (int)kd;
    ncell *= k;
    if (ncell > STATIC_MAX_CELLS) {
      set_last_error("ecmc_cells_static: more than 1048576 cells");
      return ECMC_EINVAL;
    }
    ntile *= tiles[a];
    if (ntile > INT32_MAX) {
      set_last_error("ecmc_cells_static: more than 2^31 - 1 tiles");
      return ECMC_EINVAL;
    }
    S.L[a] = box[a];
    S.nc[a] = k;
    S.cs[a] = box[a] / k;
    S.D[a] = tiles[a];
    S.T[a] = box[a] / tiles[a];
    S.W[a] = S.T[a] - joint;
    if (!(S.W[a] > 0.0)) {
      set_last_error("ecmc_cells_static: tile narrower than the joint");
      return ECMC_EINVAL;
    }
  }
  int32_t *base = nullptr;
  {
    const cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) {
      char msg[256];
      snprintf(msg, sizeof(msg), "ecmc_cells_static: looking up the scratch array failed: %s",
               cudaGetErrorString(e));
      set_last_error(msg);
      return ECMC_ECUDA;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  S.r = d_r;
  S.n = n;
  S.seed = seed;
  S.sweep = sweep;
  S.tags = d_tags;
  S.start = d_cell_start;
  S.ids = d_cell_ids;
  S.rank = base;
  S.count = base + STATIC_MAX_BEADS;
  S.bsum = base + STATIC_MAX_BEADS + STATIC_MAX_CELLS;
  // a CUDA failure of this call is reported with its code; errors are read
  // with cudaPeekAtLastError right after each launch, so an error that
  // earlier, unrelated work left on the thread is not taken for this call's
  auto failed = [](const char *what, cudaError_t e) {
    char msg[256];
    snprintf(msg, sizeof(msg), "ecmc_cells_static: %s: %s", what, cudaGetErrorString(e));
    set_last_error(msg);
    return ECMC_ECUDA;
  };
  // the counts are the only scratch that must start at zero
  cudaError_t e = cudaMemsetAsync(S.count, 0, sizeof(int32_t) * ncell, s);
  if (e != cudaSuccess) return failed("clearing the counts", e);
  const int64_t nb = (n + 255) / 256;
  const int64_t tiles_n = (ncell + ST_TILE - 1) / ST_TILE;
  ks_tag_count<<<(unsigned)nb, 256, 0, s>>>(S);
  if ((e = cudaPeekAtLastError()) != cudaSuccess) return failed("launching the tag pass", e);
  ks_scan_tiles<<<(unsigned)tiles_n, ST_BLOCK, 0, s>>>(S, ncell);
  if ((e = cudaPeekAtLastError()) != cudaSuccess) return failed("launching the scan", e);
  ks_scan_sums<<<1, ST_BLOCK, 0, s>>>(S, tiles_n, ncell);
  if ((e = cudaPeekAtLastError()) != cudaSuccess) return failed("launching the scan", e);
  ks_scan_add<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(S, ncell);
  if ((e = cudaPeekAtLastError()) != cudaSuccess) return failed("launching the scan", e);
  ks_scatter<<<(unsigned)nb, 256, 0, s>>>(S);
  if ((e = cudaPeekAtLastError()) != cudaSuccess) return failed("launching the scatter", e);
  if (shift_out) {
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)sweep, 0, 0, seed, 0);
    for (int a = 0; a < 3; ++a) shift_out[a] = unit53(w.v[a]) * S.T[a];
  }
  return ECMC_OK;
}
