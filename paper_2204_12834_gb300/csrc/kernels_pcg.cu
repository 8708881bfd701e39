// Preconditioned conjugate gradients on the reduced camera system (Sec. 4.2, eqs. `Sx`,
// `Schur`) -- the solvers the paper compares against -- built from the same matvec kernels:
//   S p = U_lam p - W V_lam^-1 W^T p   (the series group kernel for W V^-1 W^T p, then
//                                       schur_camera_kernel for U_lam p - y);
//   Schur-Jacobi preconditioner (Sec. 5, Ceres' choice): the inverses of the 9x9 diagonal
//       blocks S_cc = U_lam,c - sum_l W_cl V_l^-1 W_cl^T, whose second term is summed per
//       (landmark, camera) pair in the tiles and per camera over its slot rows;
//   power-series preconditioner (the Neumann-series preconditioner of Fig. 2, "PoCG"): the
//       series solve itself, applied to the residual (host side).
// Vector reductions use a fixed order (per-block partial sums, then one block), so the
// iterates are reproducible.
#include "poba_internal.cuh"
#include "series_body.cuh"
#include "tile_common.cuh"

namespace poba {

// ---------------------------------------------------------------------------------------
// Schur-Jacobi blocks.  Observation o with camera c and landmark l contributes through the pair
// (c, l): B = sum over the pair's observations of J_l^T J_p (3x9; a camera may observe a
// landmark more than once), C = B^T V_l^-1 B (9x9).  The first observation of each pair (pairs
// are contiguous: observations are sorted by landmark, then camera) computes C; the per-slot
// sums of C go to partial rows (stride kLinVals, entries 0..44 packed).
template <int IDX>
__device__ __forceinline__ double pair_entry(const double (&B)[27], const double (&G)[27]) {
  constexpr int a = packed_row(IDX), b = packed_col(IDX);
  return B[a] * G[b] + B[9 + a] * G[9 + b] + B[18 + a] * G[18 + b];
}

template <int R, typename T>
__device__ __forceinline__ void sj_round(bool active, bool head, int pos, const double (&B)[27],
                                         const double (&G)[27], T (*sg)[9], int ns, int n,
                                         const uint16_t* sbeg, const int* srow, T* partial) {
  if (active) {
    sg[pos][0] = head ? (T)pair_entry<R * 9 + 0>(B, G) : (T)0;
    sg[pos][1] = head ? (T)pair_entry<R * 9 + 1>(B, G) : (T)0;
    sg[pos][2] = head ? (T)pair_entry<R * 9 + 2>(B, G) : (T)0;
    sg[pos][3] = head ? (T)pair_entry<R * 9 + 3>(B, G) : (T)0;
    sg[pos][4] = head ? (T)pair_entry<R * 9 + 4>(B, G) : (T)0;
    sg[pos][5] = head ? (T)pair_entry<R * 9 + 5>(B, G) : (T)0;
    sg[pos][6] = head ? (T)pair_entry<R * 9 + 6>(B, G) : (T)0;
    sg[pos][7] = head ? (T)pair_entry<R * 9 + 7>(B, G) : (T)0;
    sg[pos][8] = head ? (T)pair_entry<R * 9 + 8>(B, G) : (T)0;
  }
  __syncthreads();
  slot_sums<T, T>(sg, ns, n, sbeg, srow, partial + R * 9, kLinVals);
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kTileObs) schur_jacobi_tile_kernel(
    Topology tp, const T* __restrict__ J, const double* __restrict__ Vinv,
    T* __restrict__ partial) {
  __shared__ T sg[kTileObs][9];
  __shared__ uint16_t sbeg[kTileObs];
  __shared__ int srow[kTileObs];
  const int tid = threadIdx.x;
  const TileHdr th = load_tile(tp, blockIdx.x);
  const int o0 = th.o0, n = th.n, ns = th.ns;
  for (int i = tid; i < ns; i += blockDim.x) {
    sbeg[i] = tp.slot_beg[th.S0 + i];
    srow[i] = tp.slot_row[th.S0 + i];
  }
  const size_t pad = (size_t)tp.n_obs_pad;
  const bool active = tid < n;
  bool head = false;
  int pos = 0;
  double B[27], G[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) B[q] = G[q] = 0.0;
  if (active) {
    const int o = o0 + tid;
    const int c = tp.cam_of[o], l = tp.lm_of[o];
    pos = tp.obs_meta[o] & 0xff;
    head = tid == 0 || tp.cam_of[o - 1] != c || tp.lm_of[o - 1] != l;
    if (head) {
      for (int q = o; q < o0 + n && tp.cam_of[q] == c && tp.lm_of[q] == l; ++q) {
        double jp[18], jl[6];
#pragma unroll
        for (int e = 0; e < 18; ++e) jp[e] = (double)J[jidx<T>(e, q, pad)];
#pragma unroll
        for (int e = 0; e < 6; ++e) jl[e] = (double)J[jidx<T>(18 + e, q, pad)];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int j = 0; j < 9; ++j) B[k * 9 + j] += jl[k] * jp[j] + jl[3 + k] * jp[9 + j];
      }
      const double* vi = Vinv + (size_t)l * 6;
      const double v0 = vi[0], v1 = vi[1], v2 = vi[2], v3 = vi[3], v4 = vi[4], v5 = vi[5];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const double b0 = B[j], b1 = B[9 + j], b2 = B[18 + j];
        G[j] = v0 * b0 + v1 * b1 + v2 * b2;
        G[9 + j] = v1 * b0 + v3 * b1 + v4 * b2;
        G[18 + j] = v2 * b0 + v4 * b1 + v5 * b2;
      }
    }
  }
  __syncthreads();
  sj_round<0>(active, head, pos, B, G, sg, ns, n, sbeg, srow, partial);
  sj_round<1>(active, head, pos, B, G, sg, ns, n, sbeg, srow, partial);
  sj_round<2>(active, head, pos, B, G, sg, ns, n, sbeg, srow, partial);
  sj_round<3>(active, head, pos, B, G, sg, ns, n, sbeg, srow, partial);
  sj_round<4>(active, head, pos, B, G, sg, ns, n, sbeg, srow, partial);
}

template <typename T>
void launch_schur_jacobi_tiles(const Topology& tp, const T* J, const double* Vinv, T* partial,
                               cudaStream_t s) {
  schur_jacobi_tile_kernel<T><<<tp.n_tiles, kTileObs, 0, s>>>(tp, J, Vinv, partial);
}
template void launch_schur_jacobi_tiles<double>(const Topology&, const double*, const double*, double*, cudaStream_t);
template void launch_schur_jacobi_tiles<float>(const Topology&, const float*, const double*, float*, cudaStream_t);

// S45[c] = U45[c] + lam D^T D - SJ45[c] (packed 9x9 diagonal blocks of S).
__global__ void schur_diag_kernel(int n_cams, const double* __restrict__ U45,
                                  const double* __restrict__ SJ45, double lam, int mode,
                                  double* __restrict__ S45) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cams * 45) return;
  const int e = i % 45;
  int row = 0, rem = e;
  while (rem >= 9 - row) {
    rem -= 9 - row;
    ++row;
  }
  const double u = U45[i];
  S45[i] = (rem == 0 ? u + damp_diag(u, lam, mode) : u) - SJ45[i];
}

void launch_schur_diag(int n_cams, const double* U45, const double* SJ45, double lam, int mode,
                       double* S45, cudaStream_t s) {
  const int n = n_cams * 45;
  schur_diag_kernel<<<(n + 255) / 256, 256, 0, s>>>(n_cams, U45, SJ45, lam, mode, S45);
}

// ---------------------------------------------------------------------------------------
// S p, camera side: q_c = U_lam,c p_c - (sum of the camera's series partial rows, chunked as in
// camera_body).  9 threads per camera.
template <typename PT>
__global__ void __launch_bounds__(kCamBlock * 9) schur_camera_kernel(
    Topology tp, const int32_t* __restrict__ cam_ptr, const PT* __restrict__ partial, const double* __restrict__ U45, double lam,
    int mode, const double* __restrict__ p, double* __restrict__ q) {
  const int cl = threadIdx.x / 9, k = threadIdx.x - 9 * (threadIdx.x / 9);
  const int c = blockIdx.x * kCamBlock + cl;
  if (c >= tp.n_cams) return;
  const int r0 = cam_ptr[c], r1 = cam_ptr[c + 1];
  const int C = cam_chunk_rows(r1 - r0);
  double y = 0.0;
  for (int q0 = r0; q0 < r1; q0 += C) y += cam_chunk_sum(partial, q0, min(q0 + C, r1), k);
  double up = 0.0;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    double u = U45[(size_t)c * 45 + (k < j ? packed9(k, j) : packed9(j, k))];
    if (j == k) u += damp_diag(u, lam, mode);
    up += u * p[(size_t)c * 9 + j];
  }
  q[(size_t)c * 9 + k] = up - y;
}

template <typename PT>
void launch_schur_camera(const Topology& tp, const SerTopo& sp, const PT* partial,
                         const double* U45, double lam, int mode, const double* p, double* q,
                         cudaStream_t s) {
  schur_camera_kernel<PT><<<camera_blocks(tp), kCamBlock * 9, 0, s>>>(tp, sp.cam_ptr, partial, U45,
                                                                      lam, mode, p, q);
}
template void launch_schur_camera<double>(const Topology&, const SerTopo&, const double*, const double*, double, int, const double*, double*, cudaStream_t);
template void launch_schur_camera<float>(const Topology&, const SerTopo&, const float*, const double*, double, int, const double*, double*, cudaStream_t);

// Reduced right-hand side of S y = -b~: out_c = (sum of the camera's partial rows, W V^-1 b_l)
// - b_p,c.  9 threads per camera.
template <typename PT>
__global__ void __launch_bounds__(kCamBlock * 9) schur_rhs_camera_kernel(
    Topology tp, const int32_t* __restrict__ cam_ptr, const PT* __restrict__ partial, const double* __restrict__ b_p,
    double* __restrict__ out) {
  const int cl = threadIdx.x / 9, k = threadIdx.x - 9 * (threadIdx.x / 9);
  const int c = blockIdx.x * kCamBlock + cl;
  if (c >= tp.n_cams) return;
  const int r0 = cam_ptr[c], r1 = cam_ptr[c + 1];
  const int C = cam_chunk_rows(r1 - r0);
  double y = 0.0;
  for (int q0 = r0; q0 < r1; q0 += C) y += cam_chunk_sum(partial, q0, min(q0 + C, r1), k);
  out[(size_t)c * 9 + k] = y - b_p[(size_t)c * 9 + k];
}

template <typename PT>
void launch_schur_rhs_camera(const Topology& tp, const SerTopo& sp, const PT* partial,
                             const double* b_p, double* out, cudaStream_t s) {
  schur_rhs_camera_kernel<PT><<<camera_blocks(tp), kCamBlock * 9, 0, s>>>(tp, sp.cam_ptr, partial,
                                                                          b_p, out);
}
template void launch_schur_rhs_camera<double>(const Topology&, const SerTopo&, const double*, const double*, double*, cudaStream_t);
template void launch_schur_rhs_camera<float>(const Topology&, const SerTopo&, const float*, const double*, double*, cudaStream_t);

// The current term rows the tile kernel gathers: t_cam[c] = p_c (bulk precision).
template <typename PT>
__global__ void stage_term_kernel(int n_cams, const double* __restrict__ p, PT* __restrict__ t_cam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cams * 9) return;
  t_cam[(size_t)(i / 9) * kTStride + i % 9] = (PT)p[i];
}

template <typename PT>
void launch_stage_term(int n_cams, const double* p, PT* t_cam, cudaStream_t s) {
  const int n = n_cams * 9;
  stage_term_kernel<PT><<<(n + 255) / 256, 256, 0, s>>>(n_cams, p, t_cam);
}
template void launch_stage_term<double>(int, const double*, double*, cudaStream_t);
template void launch_stage_term<float>(int, const double*, float*, cudaStream_t);

// ---------------------------------------------------------------------------------------
// Vector kernels of the CG recursion (length n = 9 n_cams, float64).  Scalars live in
// sc[kPcg*]; dot products go through per-block partials and one final block (fixed order).
constexpr int kDotBlocks = kPcgDotBlocks;

__global__ void __launch_bounds__(kReduceThreads) dot_partial_kernel(int n, const double* __restrict__ a,
                                                                     const double* __restrict__ b,
                                                                     double* __restrict__ part) {
  __shared__ double sred[kReduceThreads / 32];
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * per, i1 = min(i0 + per, n);
  double acc = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += a[i] * b[i];
  const double tot = block_sum_fixed(acc, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// out = a . b into sc[slot] (two launches: partials, then one block).
void launch_dot(int n, const double* a, const double* b, double* part, double* out, cudaStream_t s) {
  dot_partial_kernel<<<kDotBlocks, kReduceThreads, 0, s>>>(n, a, b, part);
  launch_reduce_sum(part, kDotBlocks, out, 1.0, s);
}

// y += alpha p, r -= alpha q with alpha = sc[kRz] / sc[kPq].
__global__ void cg_update_kernel(int n, const double* __restrict__ sc, const double* __restrict__ p,
                                 const double* __restrict__ q, double* __restrict__ y,
                                 double* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double alpha = sc[kPcgRz] / sc[kPcgPq];
  y[i] += alpha * p[i];
  r[i] -= alpha * q[i];
}

// p = z + beta p with beta = sc[kRzNew] / sc[kRz]; then sc[kRz] = sc[kRzNew] (last block).
__global__ void cg_direction_kernel(int n, double* __restrict__ sc, const double* __restrict__ z,
                                    double* __restrict__ p, int first) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double beta = first ? 0.0 : sc[kPcgRzNew] / sc[kPcgRz];
    p[i] = z[i] + beta * p[i];
  }
}

__global__ void cg_shift_kernel(double* sc) { sc[kPcgRz] = sc[kPcgRzNew]; }

void launch_cg_update(int n, const double* sc, const double* p, const double* q, double* y,
                      double* r, cudaStream_t s) {
  cg_update_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, sc, p, q, y, r);
}

void launch_cg_direction(int n, double* sc, const double* z, double* p, int first, cudaStream_t s) {
  cg_direction_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, sc, z, p, first);
  cg_shift_kernel<<<1, 1, 0, s>>>(sc);
}

// z_c = Minv_c r_c (9x9 per camera).
__global__ void block_apply_kernel(int n_cams, const double* __restrict__ M81,
                                   const double* __restrict__ r, double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_cams * 9) return;
  const int c = i / 9, k = i - 9 * c;
  const double* m = M81 + (size_t)c * 81 + k * 9;
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < 9; ++j) acc += m[j] * r[(size_t)c * 9 + j];
  z[i] = acc;
}

void launch_block_apply(int n_cams, const double* M81, const double* r, double* z, cudaStream_t s) {
  const int n = n_cams * 9;
  block_apply_kernel<<<(n + 255) / 256, 256, 0, s>>>(n_cams, M81, r, z);
}

// dst = -src (length n).
__global__ void negate_kernel(int n, const double* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = -src[i];
}

void launch_negate(int n, const double* src, double* dst, cudaStream_t s) {
  negate_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, src, dst);
}

}  // namespace poba
