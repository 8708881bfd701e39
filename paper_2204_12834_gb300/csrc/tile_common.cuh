// Device helpers shared by the tile kernels of libpoba: fixed-order reductions.
#pragma once

#include <cstdint>

namespace poba {

// Packed index of entry (i, j), i <= j, of a symmetric 9x9 matrix stored row by row.
__host__ __device__ constexpr int packed9(int i, int j) { return i * 9 - (i * (i - 1)) / 2 + (j - i); }
__host__ __device__ constexpr int packed_row(int idx) {
  int i = 0;
  while (idx >= 9 - i) { idx -= 9 - i; ++i; }
  return i;
}
__host__ __device__ constexpr int packed_col(int idx) {
  int i = 0;
  while (idx >= 9 - i) { idx -= 9 - i; ++i; }
  return i + idx;
}

// Damping of a diagonal entry d (reading of D: D^T D = diag(J^T J) clamped to [1e-6, 1e32] in
// mode 0, D = I in mode 1).
constexpr double kDampMin = 1e-6, kDampMax = 1e32;

__device__ __forceinline__ double damp_diag(double d, double lam, int mode) {
  return mode == 0 ? lam * fmin(fmax(d, kDampMin), kDampMax) : lam;
}

// Sum of `val` over the block in a fixed order (warp shuffles, then warps in order).  Must be
// called by every thread of the block; the total is valid in thread 0.  sred holds one
// double per warp.
__device__ __forceinline__ double block_sum_fixed(double val, double* sred) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sred[warp] = val;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) tot += sred[w];
  }
  return tot;
}

// Sum of `val` over a tile block in a fixed order with few FP64 instructions: the values are
// staged in sbuf ([blockDim.x] doubles), lane j of warp 0 adds values j, j + 32, j + 64, ... in
// that order, then a shuffle tree adds the lanes.  About 12 FP64 warp instructions instead of a
// shuffle tree in every warp.  Must be called by every thread of the block; the total is valid
// in thread 0.
__device__ __forceinline__ double block_sum_tile(double val, double* sbuf) {
  sbuf[threadIdx.x] = val;
  __syncthreads();
  double a = 0.0;
  if (threadIdx.x < 32) {
    a = sbuf[threadIdx.x];
    for (int j = threadIdx.x + 32; j < (int)blockDim.x; j += 32) a += sbuf[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
  }
  return a;
}

// Per-slot sums of a tile: rows sg[beg_s .. end_s) of the camera-sorted staging array are
// summed for each slot s and component k (9 per row) and written to
// out[row[s] * stride + k] (row: the slot's camera-major row, staged in shared memory).
// Small tiles split each sum over 2, 4 or 8 lanes (combined by shuffles); the split depends
// only on the slot count, so the order of every sum is fixed for a given problem.  Must be
// called by every thread of the block.
template <typename T, typename PT>
__device__ __forceinline__ void slot_sums(const T (*sg)[9], int ns, int n, const uint16_t* sbeg,
                                          const int* row, PT* out, int stride) {
  const int pairs = ns * 9;
  const int nthreads = blockDim.x;
  int split = 1;
  if (pairs * 8 <= nthreads) split = 8;
  else if (pairs * 4 <= nthreads) split = 4;
  else if (pairs * 2 <= nthreads) split = 2;
  const int total = pairs * split;
  const int bound = (total + 31) & ~31;
  for (int idx = threadIdx.x; idx < bound; idx += nthreads) {
    const int pair = idx / split, part = idx - pair * split;
    const bool act = pair < pairs;
    T acc = (T)0;
    int s = 0, k = 0;
    if (act) {
      s = pair / 9;
      k = pair - s * 9;
      const int beg = sbeg[s], end = (s + 1 < ns) ? (int)sbeg[s + 1] : n;
      for (int q = beg + part; q < end; q += split) acc += sg[q][k];
    }
    for (int off = split >> 1; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (act && part == 0) out[(size_t)row[s] * stride + k] = (PT)acc;
  }
}

}  // namespace poba
