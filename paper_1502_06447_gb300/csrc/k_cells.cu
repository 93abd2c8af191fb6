// Domain assignment and cell list (arXiv:1502.06447, Sec. II.A).
//
// Per sweep: the tile shift o in [0,T)^3 is drawn from Philox (tag 2,
// counter (2, sweep, 0, 0)); along each axis tile k covers
// [o + kT, o + (k+1)T - w) and the remaining width w is joint, whose beads
// cannot move this sweep.  The same pass bins every bead into the global
// cell grid (counting sort: count with atomics, exclusive scan, scatter of
// positions/ids/tiles into cell order).  The order of beads inside one cell
// is not fixed; nothing downstream depends on it (the EC kernel sorts what
// it stages by bead id).  With bead springs a bead whose bonded bead is
// motile in another tile is made immotile too (a spring has no longest
// bond, so only this keeps tiles apart).
#include <cuda_runtime.h>

#include "ecmc_dev.cuh"
#include "ecmc_internal.h"

namespace ecmc {
namespace {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;  // elements per thread
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__global__ void k_tag_count(const CellParams C) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n) return;
  const double r0 = C.r[3 * b], r1 = C.r[3 * b + 1], r2 = C.r[3 * b + 2];
  if (C.domain) {
    const int64_t sweep = C.sweep_dev ? *C.sweep_dev : C.sweep;
    const u64x4 w = philox(TAG_SHIFT, (uint64_t)sweep, 0, 0, C.seed, C.replica);
    const double rr[3] = {r0, r1, r2};
    int k[3];
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double o = unit53(w.v[a]) * C.T[a];
      double u = rr[a] - o;
      if (u < 0.0) u = u + C.L[a];
      if (u >= C.L[a]) u = u - C.L[a];
      int t = (int)(u / C.T[a]);
      if (t > C.D[a] - 1) t = C.D[a] - 1;
      const double loc = u - (double)t * C.T[a];
      in = in && (loc < C.W[a]);
      k[a] = t;
    }
    C.tag[b] = in ? (k[2] * C.D[1] + k[1]) * C.D[0] + k[0] : -1;
  } else {
    C.tag[b] = 0;
  }
  int c[3];
  const double rr[3] = {r0, r1, r2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int t = (int)(rr[a] / C.cs[a]);
    if (t >= C.nc[a]) t = C.nc[a] - 1;
    if (t < 0) t = 0;
    c[a] = t;
  }
  const int cell = (c[2] * C.nc[1] + c[1]) * C.nc[0] + c[0];
  C.cell[b] = cell;
  C.rank[b] = atomicAdd(&C.count[cell], 1);
}

// block-wide exclusive scan of SCAN_TILE ints; returns the tile total
__device__ int block_scan(int (&v)[SCAN_ITEMS], int *sh) {
  int local = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
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
    int w = lane < (SCAN_BLOCK / 32) ? sh[lane] : 0;
    int wi = w;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, off);
      if (lane >= off) wi += y;
    }
    if (lane < (SCAN_BLOCK / 32)) sh[lane] = wi - w;
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  const int base = sh[wid] + inc - local;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] += base;
  const int total = sh[32];
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tiles(const int *in, int64_t n, int *out,
                                                          int *block_sums) {
  __shared__ int sh[33];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < n) ? in[base + i] : 0;
  const int total = block_scan(v, sh);
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) out[base + i] = v[i];
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// exclusive scan of the block sums (one block, loops over chunks)
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(int *sums, int64_t nb, int *total_out) {
  __shared__ int sh[33];
  int carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += SCAN_TILE) {
    const int64_t base = c0 + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < nb) ? sums[base + i] : 0;
    const int total = block_scan(v, sh);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
      if (base + i < nb) sums[base + i] = v[i] + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int *out, int64_t n, const int *sums) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / SCAN_TILE];
}

__global__ void k_scatter(const CellParams C) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n) return;
  const int64_t pos = (int64_t)C.start[C.cell[b]] + C.rank[b];
  const double x = C.r[3 * b], y = C.r[3 * b + 1], z = C.r[3 * b + 2];
  C.cr[3 * pos] = x;
  C.cr[3 * pos + 1] = y;
  C.cr[3 * pos + 2] = z;
  C.crf[3 * pos] = (float)x;
  C.crf[3 * pos + 1] = (float)y;
  C.crf[3 * pos + 2] = (float)z;
  C.rf[3 * b] = (float)x;
  C.rf[3 * b + 1] = (float)y;
  C.rf[3 * b + 2] = (float)z;
  C.cid[pos] = (int32_t)b;
  int32_t t = C.tag[b];
  if (C.spring && t >= 0) {
    // bead-spring chains: a bead whose bonded bead is motile in another
    // tile waits for a later sweep (the tags of both are the ones
    // k_tag_count assigned, before any is dropped)
    const int64_t c = b % C.N;
    const int32_t tp = c != 0 ? C.tag[b - 1] : -1;
    const int32_t tn = c != C.N - 1 ? C.tag[b + 1] : -1;
    if ((tp >= 0 && tp != t) || (tn >= 0 && tn != t)) t = -1;
  }
  C.ctag[pos] = t;
  if (C.ftag) C.ftag[b] = t;
}

__global__ void k_tag_count_b(const CellBatch C) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n) return;
  const RepParams &R = C.reps[C.rep_of[b]];
  const double rr[3] = {C.r[3 * b], C.r[3 * b + 1], C.r[3 * b + 2]};
  const u64x4 w = philox(TAG_SHIFT, (uint64_t)*C.sweep_dev, 0, 0, C.seed, R.replica);
  int k[3], c[3];
  bool in = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double o = unit53(w.v[a]) * R.T[a];
    double u = rr[a] - o;
    if (u < 0.0) u = u + R.L[a];
    if (u >= R.L[a]) u = u - R.L[a];
    int t = (int)(u / R.T[a]);
    if (t > R.D[a] - 1) t = R.D[a] - 1;
    const double loc = u - (double)t * R.T[a];
    in = in && (loc < R.W[a]);
    k[a] = t;
    int q = (int)(rr[a] / R.cs[a]);
    if (q >= R.nc[a]) q = R.nc[a] - 1;
    if (q < 0) q = 0;
    c[a] = q;
  }
  C.tag[b] = in ? (k[2] * R.D[1] + k[1]) * R.D[0] + k[0] : -1;
  const int64_t cell = R.cell_off + (c[2] * R.nc[1] + c[1]) * R.nc[0] + c[0];
  C.cell[b] = (int32_t)cell;
  C.rank[b] = atomicAdd(&C.count[cell], 1);
}

__global__ void k_scatter_b(const CellBatch C) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= C.n) return;
  const int64_t pos = (int64_t)C.start[C.cell[b]] + C.rank[b];
  const double x = C.r[3 * b], y = C.r[3 * b + 1], z = C.r[3 * b + 2];
  C.cr[3 * pos] = x;
  C.cr[3 * pos + 1] = y;
  C.cr[3 * pos + 2] = z;
  C.crf[3 * pos] = (float)x;
  C.crf[3 * pos + 1] = (float)y;
  C.crf[3 * pos + 2] = (float)z;
  C.rf[3 * b] = (float)x;
  C.rf[3 * b + 1] = (float)y;
  C.rf[3 * b + 2] = (float)z;
  C.cid[pos] = (int32_t)(b - C.reps[C.rep_of[b]].bead_off);
  C.ctag[pos] = C.tag[b];
}

__global__ void k_sweep_advance(int64_t *sweep) { *sweep += 1; }

}  // namespace

cudaError_t launch_cells_batch(const CellBatch &C, int64_t ncell, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(C.count, 0, sizeof(int32_t) * ncell, s);
  if (e != cudaSuccess) return e;
  const int T = 256;
  const int64_t nb = (C.n + T - 1) / T;
  if (C.n > 0) k_tag_count_b<<<(unsigned)nb, T, 0, s>>>(C);
  const int64_t tiles = (ncell + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(C.count, ncell, C.start, C.block_sums);
  k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(C.block_sums, tiles, C.start + ncell);
  k_scan_add<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(C.start, ncell, C.block_sums);
  if (C.n > 0) k_scatter_b<<<(unsigned)nb, T, 0, s>>>(C);
  return cudaGetLastError();
}

cudaError_t launch_sweep_advance(int64_t *sweep_dev, cudaStream_t s) {
  k_sweep_advance<<<1, 1, 0, s>>>(sweep_dev);
  return cudaGetLastError();
}

size_t cells_scratch_ints(int64_t ncell) { return (size_t)((ncell + SCAN_TILE - 1) / SCAN_TILE) + 1; }

cudaError_t launch_cells(const CellParams &C, int64_t ncell, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(C.count, 0, sizeof(int32_t) * ncell, s);
  if (e != cudaSuccess) return e;
  const int T = 256;
  const int64_t nb = (C.n + T - 1) / T;
  if (C.n > 0) k_tag_count<<<(unsigned)nb, T, 0, s>>>(C);
  const int64_t tiles = (ncell + SCAN_TILE - 1) / SCAN_TILE;
  k_scan_tiles<<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(C.count, ncell, C.start, C.block_sums);
  k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(C.block_sums, tiles, C.start + ncell);
  k_scan_add<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(C.start, ncell, C.block_sums);
  if (C.n > 0) k_scatter<<<(unsigned)nb, T, 0, s>>>(C);
  return cudaGetLastError();
}

}  // namespace ecmc
