// Allocation-free cost evaluation (ba_cost_noalloc).
//
// Some callers cannot let a library call cudaMalloc: cudaMalloc / cudaFree synchronise the
// whole device, which a latency-bound loop cannot afford, and processes whose device memory is
// owned by another allocator (a framework's caching allocator, or a fixed budget handed out
// up front) must not take memory behind that allocator's back.  For them this file provides a
// variant of the float64 cost evaluation whose scratch (per-camera rotation records and
// per-block partial sums) lives in one file-scope __device__ array of fixed size.  Every GPU
// that loads the library holds that array until the process exits.
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/poba.h"
#include "poba_internal.cuh"
#include "tile_common.cuh"

namespace poba {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr int kNoAllocThreads = 256;
constexpr size_t kNoAllocPrepDoubles = (size_t)BA_NOALLOC_MAX_CAMS * kCamPrep;
constexpr size_t kNoAllocDoubles = kNoAllocPrepDoubles + kNoAllocMaxBlocks;

// The scratch: [camera records: BA_NOALLOC_MAX_CAMS x 25 doubles][block sums: 2048 doubles].
// In host code this name is only a stand-in for the device array; the kernels receive its
// device address from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// F = 1/2 sum_o w_o ||r_o||^2 with observations in the caller's order and weights w (not their
// square roots).  An index outside its range makes the sum NaN instead of reading out of
// bounds.
__global__ void __launch_bounds__(kNoAllocThreads) cost_noalloc_kernel(
    int n_cams, int n_lms, int n_obs, const double* __restrict__ prep,
    const double* __restrict__ lms, const double2* __restrict__ obs,
    const int32_t* __restrict__ cam_idx, const int32_t* __restrict__ lm_idx,
    const double* __restrict__ weights, double* __restrict__ block_sums) {
  __shared__ double sred[kNoAllocThreads / 32];
  double acc = 0.0;
  // 64-bit index: n_obs may come within one grid's stride of INT_MAX
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_obs; o += stride) {
    const int c = cam_idx[o], l = lm_idx[o];
    if (c < 0 || c >= n_cams || l < 0 || l >= n_lms) {
      acc += NAN;
      continue;
    }
    const double* q = prep + (size_t)c * kCamPrep;
    const double X0 = lms[(size_t)l * 3 + 0], X1 = lms[(size_t)l * 3 + 1], X2 = lms[(size_t)l * 3 + 2];
    const double P0 = q[0] * X0 + q[1] * X1 + q[2] * X2 + q[18];
    const double P1 = q[3] * X0 + q[4] * X1 + q[5] * X2 + q[19];
    const double P2 = q[6] * X0 + q[7] * X1 + q[8] * X2 + q[20];
    const double px = -P0 / P2, py = -P1 / P2;
    const double n2 = px * px + py * py;
    const double rad = 1.0 + n2 * (q[22] + q[23] * n2);
    const double2 ob = obs[o];
    const double r0 = q[21] * rad * px - ob.x, r1 = q[21] * rad * py - ob.y;
    double e = r0 * r0 + r1 * r1;
    if (weights) e *= weights[o];
    acc += e;
  }
  const double tot = block_sum_fixed(acc, sred);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

namespace {
ba_status reject(ba_status s, const std::string& why) {
  set_last_error(why);
  return s;
}
}  // namespace

}  // namespace poba

extern "C" {

ba_status ba_cost_noalloc(int32_t n_cams, int32_t n_lms, int32_t n_obs, const double* cams,
                          const double* lms, const double* obs, const int32_t* cam_idx,
                          const int32_t* lm_idx, const double* weights, double* cost_out,
                          void* cuda_stream) {
  using namespace poba;
  if (n_cams < 1 || n_lms < 1 || n_obs < 0)
    return reject(BA_ERR_INVALID_ARG, "ba_cost_noalloc: need n_cams >= 1, n_lms >= 1, n_obs >= 0");
  if (n_cams > BA_NOALLOC_MAX_CAMS)
    return reject(BA_ERR_INVALID_ARG, "ba_cost_noalloc: n_cams = " + std::to_string(n_cams) +
                                          " exceeds the fixed scratch limit of " +
                                          std::to_string(BA_NOALLOC_MAX_CAMS) + " cameras");
  if (!cams || !lms || !cost_out) return reject(BA_ERR_INVALID_ARG, "ba_cost_noalloc: NULL pointer");
  if (n_obs > 0 && (!obs || !cam_idx || !lm_idx))
    return reject(BA_ERR_INVALID_ARG, "ba_cost_noalloc: NULL observation pointer");
  if (((uintptr_t)obs) % 16 != 0)
    return reject(BA_ERR_INVALID_ARG, "ba_cost_noalloc: obs must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // The scratch array's address in the current device's context, looked up on every call (no
  // cache: a context that was reset and re-created holds the array at a new address).
  void* ptr = nullptr;
  const cudaError_t ea = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (ea != cudaSuccess || !ptr) {
    cudaGetLastError();
    return reject(BA_ERR_CUDA, std::string("ba_cost_noalloc: cudaGetSymbolAddress: ") +
                                   cudaGetErrorString(ea));
  }
  double* scratch = (double*)ptr;
  double* prep = scratch;
  double* block_sums = scratch + kNoAllocPrepDoubles;

  // Every scratch entry the kernels read is written earlier in the same call (camera records
  // for all n_cams cameras, one partial per launched block), so nothing needs clearing.
  launch_cam_prepare(cams, nullptr, n_cams, prep, nullptr, s);
  const int64_t want = ((int64_t)n_obs + kNoAllocThreads - 1) / kNoAllocThreads;
  const int blocks = want < 1 ? 1 : (want > kNoAllocMaxBlocks ? kNoAllocMaxBlocks : (int)want);
  cost_noalloc_kernel<<<blocks, kNoAllocThreads, 0, s>>>(n_cams, n_lms, n_obs, prep, lms,
                                                         (const double2*)obs, cam_idx, lm_idx,
                                                         weights, block_sums);
  launch_reduce_sum(block_sums, blocks, cost_out, 0.5, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return reject(BA_ERR_CUDA, std::string("ba_cost_noalloc: launch: ") + cudaGetErrorString(e));
  return BA_OK;
}

}  // extern "C"
