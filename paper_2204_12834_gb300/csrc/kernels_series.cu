// Per-term power-series kernels of libpoba (sm_103a), Sec. 4.3, and the LM helper kernels.
//
// One series term is two launches: series_group_kernel (the group body of series_body.cuh, one
// block per group of the series schedule) and camera_step_kernel (the camera body over all
// cameras, then the stop rule of eq. `qcriterion` in the last block to finish, which raises
// `done` so that later launches return at once).  These launches are what the captured-graph
// path replays; the persistent kernel in kernels_persistent.cu runs the same bodies in one
// launch.  Back-substitution (Sec. 4.2) runs over the tile schedule and also accumulates the
// model decrease 1/2||r||^2 - 1/2||r + J_p dx_p + J_l dx_l||^2.
#include <cfloat>
#include <cmath>

#include "poba_internal.cuh"
#include "series_body.cuh"
#include "tile_common.cuh"

namespace poba {

// One block per group of the series schedule (the per-term forms; the persistent kernel runs
// the same group body).  Groups of problems whose series has stopped return at once.
template <typename T, int MODE>
__global__ void __launch_bounds__(kChunkObs) series_group_kernel(
    Topology tp, SerTopo sp, const T* __restrict__ J, const T* __restrict__ t_cam,
    const double* __restrict__ b_l, const T* __restrict__ Vinv, T* __restrict__ partial,
    const SeriesState* __restrict__ st, const SeriesGlobal* __restrict__ sgl) {
  extern __shared__ __align__(16) unsigned char group_smem[];
  GroupSmem<T>& sm = *reinterpret_cast<GroupSmem<T>*>(group_smem);
  if (MODE == kModeSeries && sgl->all_done) return;
  if (st[__ldg(sp.group + 2 * blockIdx.x + 1).y].done) return;
  group_body<T, MODE>(tp, sp, blockIdx.x, J, t_cam, b_l, Vinv, partial, sm);
}

template <typename T>
cudaError_t series_group_kernels_init() {
  const int bytes = (int)sizeof(GroupSmem<T>);
  cudaError_t e = cudaFuncSetAttribute(series_group_kernel<T, kModeSeries>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(series_group_kernel<T, kModeRhs>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}
template cudaError_t series_group_kernels_init<float>();
template cudaError_t series_group_kernels_init<double>();

template <typename T>
void launch_tile_rhs(const Topology& tp, const SerTopo& sp, const T* J, const double* b_l,
                     const T* Vinv, T* partial, const SeriesState* st, cudaStream_t s) {
  if (sp.n_groups == 0) return;
  series_group_kernel<T, kModeRhs><<<sp.n_groups, kChunkObs, sizeof(GroupSmem<T>), s>>>(
      tp, sp, J, nullptr, b_l, Vinv, partial, st, nullptr);
}

template <typename T>
void launch_tile_series(const Topology& tp, const SerTopo& sp, const T* J, const T* t_cam,
                        const T* Vinv, T* partial, const SeriesState* st, const SeriesGlobal* sgl,
                        cudaStream_t s) {
  if (sp.n_groups == 0) return;
  series_group_kernel<T, kModeSeries><<<sp.n_groups, kChunkObs, sizeof(GroupSmem<T>), s>>>(
      tp, sp, J, t_cam, nullptr, Vinv, partial, st, sgl);
}

// ---------------------------------------------------------------------------------------
// Back-substitution dx_l = -V^-1 (b_l + W^T dx_p) and the model decrease per tile.
template <typename T>
__global__ void __launch_bounds__(kTileObs) tile_backsub_kernel(
    Topology tp, const T* __restrict__ J, const T* __restrict__ r, const double* __restrict__ x,
    const double* __restrict__ b_l, const T* __restrict__ Vinv, double* __restrict__ dx_l,
    double* __restrict__ block_pred) {
  __shared__ T tcam[kTileObs][9];
  __shared__ T sv[kTileObs][3];
  __shared__ double sred[kTileObs];

  const int tile = blockIdx.x, tid = threadIdx.x;
  const TileHdr th = load_tile(tp, tile);
  const int L0 = th.L0, L1 = th.L0 + th.nl, o0 = th.o0, n = th.n, S0 = th.S0, ns = th.ns;
  if (tp.n_long > 0 && tp.lm_long[L0] >= 0) return;  // a piece of a long track (below)
  for (int i = tid; i < ns * 9; i += blockDim.x) {
    const int s = i / 9, k = i - s * 9;
    int c = tp.slot_cam[S0 + s];
    POBA_CHK(tp.chk, c, tp.n_cams, kChkBackCam);
    tcam[s][k] = (T)x[(size_t)c * 9 + k];
  }
  __syncthreads();
  const bool active = tid < n;
  const size_t pad = (size_t)tp.n_obs_pad;
  T jp[18], jl[6];
  T u0 = (T)0, u1 = (T)0;
  if (active) {
    const int o = o0 + tid;
    const int meta = tp.obs_meta[o];
    load_J(J, pad, o, jp, jl);
    int sl = meta >> 8;
    POBA_CHK(tp.chk, sl, ns, kChkBackSlot);
    const T* tc = tcam[sl];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      u0 += jp[j] * tc[j];
      u1 += jp[9 + j] * tc[j];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sv[tid][k] = jl[k] * u0 + jl[3 + k] * u1;
  }
  __syncthreads();
  if (tid < L1 - L0) {
    const int l = L0 + tid;
    int a = tp.lm_seg[l] - o0, b = tp.lm_seg[l + 1] - o0;
    if (kChecks && (a < 0 || b < a || b > n)) {
      int bad = b > n ? b : a;
      POBA_CHK(tp.chk, bad, 0, kChkBackSeg);
      a = b = 0;
    }
    T s[3] = {(T)b_l[(size_t)l * 3 + 0], (T)b_l[(size_t)l * 3 + 1], (T)b_l[(size_t)l * 3 + 2]};
    for (int q = a; q < b; ++q) {
      s[0] += sv[q][0];
      s[1] += sv[q][1];
      s[2] += sv[q][2];
    }
    T z[3];
    apply_vinv(Vinv + (size_t)l * 6, s, z);
    z[0] = -z[0];
    z[1] = -z[1];
    z[2] = -z[2];
    dx_l[(size_t)l * 3 + 0] = (double)z[0];
    dx_l[(size_t)l * 3 + 1] = (double)z[1];
    dx_l[(size_t)l * 3 + 2] = (double)z[2];
    for (int q = a; q < b; ++q) {
      sv[q][0] = z[0];
      sv[q][1] = z[1];
      sv[q][2] = z[2];
    }
  }
  __syncthreads();
  double pred = 0.0;
  if (active) {
    const int o = o0 + tid;
    const T z0 = sv[tid][0], z1 = sv[tid][1], z2 = sv[tid][2];
    const double r0 = (double)r[o], r1 = (double)r[pad + o];
    const double q0 = r0 + (double)u0 + (double)(jl[0] * z0 + jl[1] * z1 + jl[2] * z2);
    const double q1 = r1 + (double)u1 + (double)(jl[3] * z0 + jl[4] * z1 + jl[5] * z2);
    pred = (r0 * r0 + r1 * r1) - (q0 * q0 + q1 * q1);
  }
  const double tot = block_sum_tile(pred, sred);
  if (tid == 0) block_pred[tile] = tot;
}

// Back-substitution of a long track (one block per track): dx_l = -V^-1 (b_l + sum over
// every observation of J_l^T J_p x_c), each piece's sum in a fixed order (block_sum_tile, in
// double) and the pieces added in order; every piece receives dx_l.  Then each piece's model
// decrease terms (as in the tile kernel) are summed into block_pred of the piece's tile.
template <typename T>
__global__ void __launch_bounds__(kTileObs) long_backsub_kernel(
    Topology tp, const T* __restrict__ J, const T* __restrict__ r, const double* __restrict__ x,
    const double* __restrict__ b_l, const T* __restrict__ Vinv, double* __restrict__ dx_l,
    double* __restrict__ block_pred) {
  __shared__ double sbuf[kTileObs];
  __shared__ double zs[3];
  const int j = blockIdx.x, tid = threadIdx.x;
  const int l0 = tp.long_first[j], np = tp.long_np[j], t0 = tp.long_tile0[j];
  const size_t pad = (size_t)tp.n_obs_pad;
  auto obs_u = [&](int o, T (&jp)[18], T (&jl)[6], T& u0, T& u1) {
    const int c = tp.cam_of[o];
    load_J(J, pad, o, jp, jl);
    u0 = (T)0;
    u1 = (T)0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const T xk = (T)x[(size_t)c * 9 + k];
      u0 += jp[k] * xk;
      u1 += jp[9 + k] * xk;
    }
  };
  double S0 = 0.0, S1 = 0.0, S2 = 0.0;
  for (int q = 0; q < np; ++q) {
    const int o0 = tp.lm_seg[l0 + q];
    int n = tp.lm_seg[l0 + q + 1] - o0;
    POBA_CHK(tp.chk, n, kTileObs + 1, kChkLongSeg);
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (tid < n) {
      T jp[18], jl[6], u0, u1;
      obs_u(o0 + tid, jp, jl, u0, u1);
      v0 = (double)(jl[0] * u0 + jl[3] * u1);
      v1 = (double)(jl[1] * u0 + jl[4] * u1);
      v2 = (double)(jl[2] * u0 + jl[5] * u1);
    }
    const double a0 = block_sum_tile(v0, sbuf);
    __syncthreads();
    const double a1 = block_sum_tile(v1, sbuf);
    __syncthreads();
    const double a2 = block_sum_tile(v2, sbuf);
    __syncthreads();
    S0 += a0;
    S1 += a1;
    S2 += a2;
  }
  if (tid == 0) {
    const double s0 = b_l[(size_t)l0 * 3 + 0] + S0, s1 = b_l[(size_t)l0 * 3 + 1] + S1,
                 s2 = b_l[(size_t)l0 * 3 + 2] + S2;
    const T* vi = Vinv + (size_t)l0 * 6;
    const double w0 = (double)vi[0], w1 = (double)vi[1], w2 = (double)vi[2];
    const double w3 = (double)vi[3], w4 = (double)vi[4], w5 = (double)vi[5];
    zs[0] = -(w0 * s0 + w1 * s1 + w2 * s2);
    zs[1] = -(w1 * s0 + w3 * s1 + w4 * s2);
    zs[2] = -(w2 * s0 + w4 * s1 + w5 * s2);
  }
  __syncthreads();
  for (int q = tid; q < np; q += blockDim.x) {
    dx_l[(size_t)(l0 + q) * 3 + 0] = zs[0];
    dx_l[(size_t)(l0 + q) * 3 + 1] = zs[1];
    dx_l[(size_t)(l0 + q) * 3 + 2] = zs[2];
  }
  const T z0 = (T)zs[0], z1 = (T)zs[1], z2 = (T)zs[2];
  for (int q = 0; q < np; ++q) {
    const int o0 = tp.lm_seg[l0 + q], n = tp.lm_seg[l0 + q + 1] - o0;
    double pred = 0.0;
    if (tid < n) {
      const int o = o0 + tid;
      T jp[18], jl[6], u0, u1;
      obs_u(o, jp, jl, u0, u1);
      const double r0 = (double)r[o], r1 = (double)r[pad + o];
      const double q0 = r0 + (double)u0 + (double)(jl[0] * z0 + jl[1] * z1 + jl[2] * z2);
      const double q1 = r1 + (double)u1 + (double)(jl[3] * z0 + jl[4] * z1 + jl[5] * z2);
      pred = (r0 * r0 + r1 * r1) - (q0 * q0 + q1 * q1);
    }
    const double tot = block_sum_tile(pred, sbuf);
    if (tid == 0) block_pred[t0 + q] = tot;
    __syncthreads();
  }
}

// Debug builds: guard bytes after the sub-buffers of an allocation (block i checks the
// kCanaryBytes bytes at offset off[i]); a changed byte records site site0 + i.
__global__ void __launch_bounds__(kCanaryBytes) canary_check_kernel(
    const uint8_t* __restrict__ base, const uint64_t* __restrict__ off, int n, unsigned site0,
    CheckRecord* chk) {
  const int i = blockIdx.x;
  if (i >= n) return;
  const uint64_t at = off[i] + threadIdx.x;
  const unsigned char v = base[at];
  if (v != kCanaryByte) {
    if (atomicCAS(&chk->site, 0u, site0 + (unsigned)i) == 0u) {
      chk->index = (long long)at;
      chk->bound = (long long)v;
    }
    atomicAdd(&chk->count, 1u);
  }
}

void launch_canary_check(const uint8_t* base, const uint64_t* off, int n, unsigned site0,
                         CheckRecord* chk, cudaStream_t s) {
  if (n > 0) canary_check_kernel<<<n, kCanaryBytes, 0, s>>>(base, off, n, site0, chk);
}

template <typename T>
void launch_tile_backsub(const Topology& tp, const T* J, const T* r, const double* x,
                         const double* b_l, const T* Vinv, double* dx_l, double* block_pred,
                         cudaStream_t s) {
  tile_backsub_kernel<T><<<tp.n_tiles, kTileObs, 0, s>>>(tp, J, r, x, b_l, Vinv, dx_l, block_pred);
  if (tp.n_long > 0)
    long_backsub_kernel<T><<<tp.n_long, kTileObs, 0, s>>>(tp, J, r, x, b_l, Vinv, dx_l, block_pred);
}

template void launch_tile_rhs<double>(const Topology&, const SerTopo&, const double*, const double*, const double*, double*, const SeriesState*, cudaStream_t);
template void launch_tile_rhs<float>(const Topology&, const SerTopo&, const float*, const double*, const float*, float*, const SeriesState*, cudaStream_t);
template void launch_tile_series<double>(const Topology&, const SerTopo&, const double*, const double*, const double*, double*, const SeriesState*, const SeriesGlobal*, cudaStream_t);
template void launch_tile_series<float>(const Topology&, const SerTopo&, const float*, const float*, const float*, float*, const SeriesState*, const SeriesGlobal*, cudaStream_t);
template void launch_tile_backsub<double>(const Topology&, const double*, const double*, const double*, const double*, const double*, double*, double*, cudaStream_t);
template void launch_tile_backsub<float>(const Topology&, const float*, const float*, const double*, const double*, const float*, double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------------------
int camera_blocks(const Topology& tp) { return (tp.n_cams + kCamBlock - 1) / kCamBlock; }

// Camera step: CS cameras x 9 components per block (camera body, norm pair per camera), then
// the stop rule of every running problem in the last block to finish.  A handle with one or two
// problems takes 8-camera blocks, which spread the latency-bound row sums over many SMs; a batch
// takes kCamBlock cameras (9 warps), so that the last block has warps for its many problems.
template <typename PT, int MODE, int CS>
__global__ void __launch_bounds__(CS * 9) camera_step_kernel(
    Topology tp, const int32_t* __restrict__ cam_ptr, const PT* __restrict__ partial,
    const double* __restrict__ b_p,
    const double* __restrict__ Uinv, double* __restrict__ x, PT* __restrict__ t_cam,
    double* __restrict__ cam_norm, SeriesState* __restrict__ st, SeriesGlobal* __restrict__ sgl,
    int iter, double eps) {
  __shared__ double ys[CS][9];
  __shared__ double y2[CS][9];
  __shared__ int is_last, s_running;
  __shared__ double red[2 * kNormLanes];
  if (MODE == kModeSeries && sgl->all_done) return;
  const int tid = threadIdx.x;
  camera_body<PT, MODE>(tp, cam_ptr, blockIdx.x * CS, CS, partial, b_p, Uinv, x, t_cam, st,
                        cam_norm, ys, y2);
  if (tid == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&sgl->counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  problems_stop_rule(tp, cam_norm, st, sgl, iter, eps, &s_running, red);
  if (tid == 0) sgl->counter = 0u;
}

template <typename PT, int MODE>
void launch_camera_step(const Topology& tp, const SerTopo& sp, const PT* partial,
                        const double* b_p, const double* Uinv, double* x, PT* t_cam,
                        double* cam_norm, SeriesState* st, SeriesGlobal* sgl, int iter, double eps,
                        cudaStream_t s) {
  constexpr int kSmall = 8;
  if (tp.n_probs <= 2)
    camera_step_kernel<PT, MODE, kSmall><<<(tp.n_cams + kSmall - 1) / kSmall, kSmall * 9, 0, s>>>(
        tp, sp.cam_ptr, partial, b_p, Uinv, x, t_cam, cam_norm, st, sgl, iter, eps);
  else
    camera_step_kernel<PT, MODE, kCamBlock><<<camera_blocks(tp), kCamBlock * 9, 0, s>>>(
        tp, sp.cam_ptr, partial, b_p, Uinv, x, t_cam, cam_norm, st, sgl, iter, eps);
}

template <typename PT>
void launch_camera_rhs(const Topology& tp, const SerTopo& sp, const PT* partial, const double* b_p,
                       const double* Uinv, double* x, PT* t_cam, double* cam_norm,
                       SeriesState* st, SeriesGlobal* sgl, cudaStream_t s) {
  launch_camera_step<PT, kModeRhs>(tp, sp, partial, b_p, Uinv, x, t_cam, cam_norm, st, sgl, 0,
                                   0.0, s);
}

template <typename PT>
void launch_camera_series(const Topology& tp, const SerTopo& sp, const PT* partial,
                          const double* Uinv, double* x, PT* t_cam, double* cam_norm,
                          SeriesState* st, SeriesGlobal* sgl, int iter, double eps,
                          cudaStream_t s) {
  launch_camera_step<PT, kModeSeries>(tp, sp, partial, nullptr, Uinv, x, t_cam, cam_norm, st,
                                      sgl, iter, eps, s);
}

template void launch_camera_rhs<double>(const Topology&, const SerTopo&, const double*, const double*, const double*, double*, double*, double*, SeriesState*, SeriesGlobal*, cudaStream_t);
template void launch_camera_rhs<float>(const Topology&, const SerTopo&, const float*, const double*, const double*, double*, float*, double*, SeriesState*, SeriesGlobal*, cudaStream_t);
template void launch_camera_series<double>(const Topology&, const SerTopo&, const double*, const double*, double*, double*, double*, SeriesState*, SeriesGlobal*, int, double, cudaStream_t);
template void launch_camera_series<float>(const Topology&, const SerTopo&, const float*, const double*, double*, float*, double*, SeriesState*, SeriesGlobal*, int, double, cudaStream_t);

// ---------------------------------------------------------------------------------------
__global__ void series_reset_kernel(SeriesState* st, SeriesGlobal* sgl, const LmRecord* rec,
                                    int n_probs) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0) {
    sgl->all_done = 0;
    sgl->counter = 0u;
  }
  if (p >= n_probs) return;
  st[p].done = (rec && !rec[p].active) ? 1 : 0;
  st[p].m = 0;
  st[p].stopped = 0;
  st[p].stop_value = INFINITY;
  st[p].x_norm = 0.0;
  st[p].t_norm = 0.0;
}

void launch_series_reset(SeriesState* st, SeriesGlobal* sgl, const LmRecord* rec, int n_probs,
                         cudaStream_t s) {
  series_reset_kernel<<<(n_probs + 127) / 128, 128, 0, s>>>(st, sgl, rec, n_probs);
}

// ---------------------------------------------------------------------------------------
// State input / output between the caller's landmark order and the internal order.
__global__ void check_finite_kernel(const double* __restrict__ src, int n, int32_t* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(src[i])) atomicOr(bad, 1);
}

__global__ void gather_rows3_kernel(const double* __restrict__ src, const int32_t* __restrict__ order,
                                    int n, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) dst[i] = src[(size_t)order[i / 3] * 3 + i % 3];
}

__global__ void scatter_rows3_kernel(const double* __restrict__ src, const int32_t* __restrict__ order,
                                     int n, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * n) dst[(size_t)order[i / 3] * 3 + i % 3] = src[i];
}

// *differ |= 1 when src differs from the current state cur in any bit: src[i] against cur[i]
// (order null), or the caller-order rows src[order[r]] against the internal rows cur[r] (3 values
// per row, n rows).
__global__ void state_differs_kernel(const double* __restrict__ src, const double* __restrict__ cur,
                                     const int32_t* __restrict__ order, int n, int32_t* differ) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = order ? 3 * n : n;
  if (i >= m) return;
  const double a = order ? src[(size_t)order[i / 3] * 3 + i % 3] : src[i];
  if (__double_as_longlong(a) != __double_as_longlong(cur[i])) atomicOr(differ, 1);
}

void launch_state_differs(const double* src, const double* cur, const int32_t* order, int n,
                          int32_t* differ, cudaStream_t s) {
  const int m = order ? 3 * n : n;
  if (m > 0) state_differs_kernel<<<(m + 255) / 256, 256, 0, s>>>(src, cur, order, n, differ);
}

void launch_check_finite(const double* src, int n, int32_t* bad, cudaStream_t s) {
  if (n > 0) check_finite_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, n, bad);
}
void launch_gather_rows3(const double* src, const int32_t* order, int n, double* dst, cudaStream_t s) {
  if (n > 0) gather_rows3_kernel<<<(3 * n + 255) / 256, 256, 0, s>>>(src, order, n, dst);
}
void launch_scatter_rows3(const double* src, const int32_t* order, int n, double* dst, cudaStream_t s) {
  if (n > 0) scatter_rows3_kernel<<<(3 * n + 255) / 256, 256, 0, s>>>(src, order, n, dst);
}

__global__ void set_scalar_kernel(double* dst, double v) { *dst = v; }

void launch_set_scalar(double* dst, double v, cudaStream_t s) { set_scalar_kernel<<<1, 1, 0, s>>>(dst, v); }

// Fixed-order sum of n doubles into *out (one block).
__global__ void __launch_bounds__(kReduceThreads) reduce_sum_kernel(const double* in, int n,
                                                                     double* out, double scale) {
  __shared__ double sred[kReduceThreads / 32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += in[i];
  const double tot = block_sum_fixed(a, sred);
  if (threadIdx.x == 0) *out = scale * tot;
}

void launch_reduce_sum(const double* in, int n, double* out, double scale, cudaStream_t s) {
  reduce_sum_kernel<<<1, kReduceThreads, 0, s>>>(in, n, out, scale);
}

// One block per problem: scale * (sum of the problem's tile values), fixed order.
// v[t0] + v[t0 + stride] + ... (t < t1) added in that order, with the loads issued eight at a
// time so that the sum waits for one round trip per eight values.
__device__ __forceinline__ double strided_sum(const double* __restrict__ v, int t0, int t1,
                                              int stride) {
  double a = 0.0;
  for (int t = t0; t < t1; t += 8 * stride) {
    double buf[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) buf[j] = t + j * stride < t1 ? v[t + j * stride] : 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (t + j * stride < t1) a += buf[j];
  }
  return a;
}

__global__ void __launch_bounds__(kReduceThreads) reduce_tiles_kernel(Topology tp,
                                                                       const double* tile_vals,
                                                                       double* out, int out_stride,
                                                                       double scale) {
  __shared__ double sred[kReduceThreads / 32];
  const int p = blockIdx.x;
  const double a = strided_sum(tile_vals, tp.tile_off[p] + threadIdx.x, tp.tile_off[p + 1],
                               blockDim.x);
  const double tot = block_sum_fixed(a, sred);
  if (threadIdx.x == 0) out[(size_t)p * out_stride] = scale * tot;
}

void launch_reduce_tiles(const Topology& tp, const double* tile_vals, double* out, int out_stride,
                         double scale, cudaStream_t s) {
  reduce_tiles_kernel<<<tp.n_probs, kReduceThreads, 0, s>>>(tp, tile_vals, out, out_stride, scale);
}

// ---------------------------------------------------------------------------------------
// LM decision (Sec. 5.1), one block per problem: F(x + dx) and the model decrease from the
// problem's tile sums, gain ratio, accept iff F decreased and the model decrease is positive,
// lambda / nu update.  An iteration whose damped blocks were not positive definite has no step
// and counts as rejected (its trial cost is reported as NaN).
constexpr double kLambdaMin = 1e-10, kLambdaMax = 1e32;

__global__ void __launch_bounds__(kReduceThreads) lm_decide_kernel(
    Topology tp, const double* tile_cost, const double* tile_pred, const int32_t* not_spd,
    LmRecord* rec_all, double func_tol, int deactivate, int32_t* relin) {
  __shared__ double sred[kReduceThreads / 32];
  const int p = blockIdx.x;
  LmRecord* rec = rec_all + p;
  const int t0 = tp.tile_off[p] + threadIdx.x, t1 = tp.tile_off[p + 1];
  const double a = strided_sum(tile_cost, t0, t1, blockDim.x);
  const double b = strided_sum(tile_pred, t0, t1, blockDim.x);
  double F_new = 0.5 * block_sum_fixed(a, sred);
  __syncthreads();
  double pred = 0.5 * block_sum_fixed(b, sred);
  if (threadIdx.x != 0) return;
  if (!rec->active) {
    rec->accepted = 0;
    return;
  }
  const int bad = not_spd[p] != 0;
  if (bad) {
    F_new = NAN;
    pred = 0.0;
  }
  const double F = rec->cost;
  const double actual = F - F_new;
  const int accepted = (!bad && isfinite(F_new) && actual > 0.0 && pred > 0.0) ? 1 : 0;
  const double rho = (!bad && pred != 0.0) ? actual / pred : 0.0;
  double lam = rec->lambda, nu = rec->nu;
  rec->lambda_used = lam;
  if (accepted) {
    const double q = 2.0 * rho - 1.0;
    lam *= fmax(1.0 / 3.0, 1.0 - q * q * q);
    nu = 2.0;
  } else {
    lam *= nu;
    nu *= 2.0;
  }
  rec->lambda = fmin(fmax(lam, kLambdaMin), kLambdaMax);
  rec->nu = nu;
  rec->cost_before = F;
  rec->cost_trial = F_new;
  rec->model_decrease = pred;
  rec->gain_ratio = rho;
  rec->accepted = accepted;
  if (accepted && relin) *relin = 1;
  rec->not_spd = bad;
  rec->converged = (accepted && actual / F < func_tol) ? 1 : 0;
  rec->nonfinite = (bad || isfinite(F_new)) ? 0 : 1;
  if (accepted) rec->cost = F_new;
  rec->iteration += 1;
  if (deactivate && rec->converged) rec->active = 0;
}

void launch_lm_decide(const Topology& tp, const double* tile_cost, const double* tile_pred,
                      const int32_t* not_spd, LmRecord* rec, double func_tol, int deactivate,
                      cudaStream_t s, int32_t* relin) {
  lm_decide_kernel<<<tp.n_probs, kReduceThreads, 0, s>>>(tp, tile_cost, tile_pred, not_spd, rec,
                                                         func_tol, deactivate, relin);
}

// x <- x + dx for the problems whose step was accepted (cameras already summed in cams_trial).
__global__ void apply_step_kernel(Topology tp, const LmRecord* rec, double* cams,
                                  const double* cams_trial, double* lms, const double* dx_l) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < tp.n_cams * 9 && rec[tp.cam_prob[i / 9]].accepted) cams[i] = cams_trial[i];
  if (i < tp.n_lms * 3 && rec[tp.lm_prob[i / 3]].accepted) lms[i] += dx_l[i];
}

void launch_apply_step(const Topology& tp, const LmRecord* rec, double* cams,
                       const double* cams_trial, double* lms, const double* dx_l,
                       cudaStream_t s) {
  const int n = tp.n_cams * 9 > tp.n_lms * 3 ? tp.n_cams * 9 : tp.n_lms * 3;
  const int threads = 256;
  apply_step_kernel<<<(n + threads - 1) / threads, threads, 0, s>>>(tp, rec, cams, cams_trial, lms,
                                                                    dx_l);
}

}  // namespace poba
