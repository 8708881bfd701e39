// Linearisation-side kernels of libpoba (sm_103a):
//   cam_prepare      per camera: R(w), the rotation-derivative matrix G, t, f, k1, k2
//   linearize        per observation: BAL residual r (Sec. 4) and its Jacobians J_p (2x9),
//                    J_l (2x3) by the analytic chain rule; fused with the landmark blocks
//                    V = J_l^T J_l, b_l = J_l^T r and the per-tile camera sums of
//                    J_p^T J_p, J_p^T r (Sec. 4.1, eq. `normal`)
//   lin_camera_reduce per camera: U = J_p^T J_p (45 packed), b_p = J_p^T r across tiles
//   damp_invert      U_lambda, V_lambda (Sec. 4.1) and their Cholesky inverses in float64
//   cost             F(x) = 1/2 sum w ||r||^2 in float64 (Sec. 4), fixed-order block sums
//
// Camera model (BAL convention): P = R(w) X + t, p = -P_xy / P_z,
// pi = f (1 + k1 |p|^2 + k2 |p|^4) p, r = pi - obs.  With the left Jacobian G of SO(3),
// d(R(w) X)/dw = -[R X]x G; for |w|^2 below machine epsilon R = I + [w]x and
// d(R X)/dw = -[X]x.
#include <cfloat>
#include <cmath>

#include "jacobian_io.cuh"
#include "poba_internal.cuh"
#include "tile_common.cuh"

namespace poba {

// ---------------------------------------------------------------------------------------
__global__ void cam_prepare_kernel(const double* __restrict__ cams, const double* __restrict__ dx_p,
                                   int n_cams, double* __restrict__ prep,
                                   double* __restrict__ cams_out, float* __restrict__ prep32,
                                   const int32_t* __restrict__ gate) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cams || (gate && *gate == 0)) return;
  double p[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) p[j] = cams[c * 9 + j] + (dx_p ? dx_p[c * 9 + j] : 0.0);
  if (cams_out) {
#pragma unroll
    for (int j = 0; j < 9; ++j) cams_out[c * 9 + j] = p[j];
  }
  const double w0 = p[0], w1 = p[1], w2 = p[2];
  const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
  double R[9], G[9], first;
  if (th2 < DBL_EPSILON) {
    R[0] = 1.0; R[1] = -w2; R[2] = w1;
    R[3] = w2;  R[4] = 1.0; R[5] = -w0;
    R[6] = -w1; R[7] = w0;  R[8] = 1.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) G[j] = (j % 4 == 0) ? 1.0 : 0.0;
    first = 1.0;
  } else {
    const double th = sqrt(th2);
    double s, co;
    sincos(th, &s, &co);
    const double hs = sin(0.5 * th);
    const double omc = 2.0 * hs * hs;  // 1 - cos(th) without cancellation
    const double k0 = w0 / th, k1 = w1 / th, k2 = w2 / th;
    R[0] = co + omc * k0 * k0;      R[1] = -s * k2 + omc * k0 * k1; R[2] = s * k1 + omc * k0 * k2;
    R[3] = s * k2 + omc * k0 * k1;  R[4] = co + omc * k1 * k1;      R[5] = -s * k0 + omc * k1 * k2;
    R[6] = -s * k1 + omc * k0 * k2; R[7] = s * k0 + omc * k1 * k2;  R[8] = co + omc * k2 * k2;
    // G = I + a [w]x + b [w]x^2, a = (1 - cos th)/th^2, b = (th - sin th)/th^3;
    // [w]x^2 = w w^T - th^2 I.  b by its Taylor series for small th (cancellation).
    const double a = omc / th2;
    const double b = (th < 1e-2) ? (1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0)
                                 : (th - s) / (th2 * th);
    const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    const double ww[3] = {w0, w1, w2};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        G[i * 3 + j] = (i == j ? 1.0 - b * th2 : 0.0) + a * W[i * 3 + j] + b * ww[i] * ww[j];
    first = 0.0;
  }
  double* q = prep + (size_t)c * kCamPrep;
#pragma unroll
  for (int j = 0; j < 9; ++j) q[j] = R[j];
#pragma unroll
  for (int j = 0; j < 9; ++j) q[9 + j] = G[j];
  q[18] = p[3]; q[19] = p[4]; q[20] = p[5];
  q[21] = p[6]; q[22] = p[7]; q[23] = p[8];
  q[24] = first;
  if (prep32) {  // the FP32-bulk linearisation reads the record in float, converted once here
#pragma unroll
    for (int j = 0; j < kCamPrep; ++j) prep32[(size_t)c * kCamPrep + j] = (float)q[j];
  }
}

void launch_cam_prepare(const double* cams, const double* dx_p, int n_cams, double* prep,
                        double* cams_out, cudaStream_t s, float* prep32, const int32_t* gate) {
  // one warp per block: the FP64 rotation work (sin, cos, sqrt) spreads over many SMs
  int threads = 32, blocks = (n_cams + threads - 1) / threads;
  cam_prepare_kernel<<<blocks, threads, 0, s>>>(cams, dx_p, n_cams, prep, cams_out, prep32, gate);
}

// ---------------------------------------------------------------------------------------
// Entry e of a slot's camera contribution as two products of staged values (J_p row 0 at 0..8,
// row 1 at 9..17, r at 18, 19): packed (J_p^T J_p)_{ab} for e < 45, (J_p^T r)_j for e >= 45.
struct LinPairTable {
  uchar4 v[kLinVals];
};
__host__ __device__ constexpr LinPairTable make_lin_pairs() {
  LinPairTable t{};
  for (int e = 0; e < kLinVals; ++e) {
    if (e < 45) {
      const int a = packed_row(e), b = packed_col(e);
      t.v[e] = uchar4{(unsigned char)a, (unsigned char)b, (unsigned char)(9 + a), (unsigned char)(9 + b)};
    } else {
      const int j = e - 45;
      t.v[e] = uchar4{(unsigned char)j, 18, (unsigned char)(9 + j), 19};
    }
  }
  return t;
}
__constant__ LinPairTable kLinPairs = make_lin_pairs();

// Residual and Jacobians of one observation in precision T.
template <typename T>
__device__ __forceinline__ void bal_residual_jacobian(const T* __restrict__ q, const double X0d,
                                                      const double X1d, const double X2d,
                                                      const vec2<T> ob, T sw, T (&jp)[18],
                                                      T (&jl)[6], T (&r)[2]) {
  const T R[9] = {(T)q[0], (T)q[1], (T)q[2], (T)q[3], (T)q[4], (T)q[5], (T)q[6], (T)q[7], (T)q[8]};
  const T G[9] = {(T)q[9], (T)q[10], (T)q[11], (T)q[12], (T)q[13], (T)q[14], (T)q[15], (T)q[16], (T)q[17]};
  const T t0 = (T)q[18], t1 = (T)q[19], t2 = (T)q[20];
  const T f = (T)q[21], k1 = (T)q[22], k2 = (T)q[23];
  const bool first = q[24] != (T)0;
  const T X0 = (T)X0d, X1 = (T)X1d, X2 = (T)X2d;
  const T RX0 = R[0] * X0 + R[1] * X1 + R[2] * X2;
  const T RX1 = R[3] * X0 + R[4] * X1 + R[5] * X2;
  const T RX2 = R[6] * X0 + R[7] * X1 + R[8] * X2;
  const T P0 = RX0 + t0, P1 = RX1 + t1, P2 = RX2 + t2;
  const T Y0 = first ? X0 : RX0, Y1 = first ? X1 : RX1, Y2 = first ? X2 : RX2;
  // D = dP/dw = -[Y]x G
  T D[9];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    D[0 * 3 + j] = Y2 * G[3 + j] - Y1 * G[6 + j];
    D[1 * 3 + j] = Y0 * G[6 + j] - Y2 * G[0 + j];
    D[2 * 3 + j] = Y1 * G[0 + j] - Y0 * G[3 + j];
  }
  const T iz = (T)1 / P2;
  const T px = -P0 * iz, py = -P1 * iz;
  const T n2 = px * px + py * py;
  const T rad = (T)1 + n2 * (k1 + k2 * n2);
  const T drad = k1 + (T)2 * k2 * n2;
  // M = f (rad I + 2 drad p p^T);  A = dpi/dP = -iz M [I | p]
  const T m00 = f * (rad + (T)2 * drad * px * px);
  const T m01 = f * ((T)2 * drad * px * py);
  const T m11 = f * (rad + (T)2 * drad * py * py);
  T A[6];
  A[0] = -iz * m00; A[1] = -iz * m01; A[2] = -iz * (m00 * px + m01 * py);
  A[3] = -iz * m01; A[4] = -iz * m11; A[5] = -iz * (m01 * px + m11 * py);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      jp[i * 9 + j] = sw * (A[i * 3 + 0] * D[0 + j] + A[i * 3 + 1] * D[3 + j] + A[i * 3 + 2] * D[6 + j]);
      jp[i * 9 + 3 + j] = sw * A[i * 3 + j];
      jl[i * 3 + j] = sw * (A[i * 3 + 0] * R[0 + j] + A[i * 3 + 1] * R[3 + j] + A[i * 3 + 2] * R[6 + j]);
    }
  }
  const T pc[2] = {px, py};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    jp[i * 9 + 6] = sw * rad * pc[i];
    jp[i * 9 + 7] = sw * f * n2 * pc[i];
    jp[i * 9 + 8] = sw * f * n2 * n2 * pc[i];
  }
  r[0] = sw * (f * rad * px - (T)ob.x);
  r[1] = sw * (f * rad * py - (T)ob.y);
}

// kWeighted = false: every weight is 1, so the products by the square-root weight fold away
// (x * 1 = x exactly); they would otherwise cost about 26 FP64 operations per observation.
template <typename T, bool kWeighted>
__global__ void __launch_bounds__(kTileObs) linearize_kernel(
    Topology tp, const T* __restrict__ prep, const double* __restrict__ lms,
    const vec2<T>* __restrict__ obs, const T* __restrict__ sqrt_w, T* __restrict__ J,
    T* __restrict__ r, double* __restrict__ V, double* __restrict__ b_l, T* __restrict__ partial,
    double* __restrict__ block_cost, const int32_t* __restrict__ gate) {
  // sj: J_p and r of each observation at its camera-sorted position; s9: the landmark
  // contributions.  In FP64 the two share storage (the static limit is 48 KB), with a barrier
  // between the landmark sums and the staging.
  // sj rows hold 20 values with a stride of 21 (odd), so that the threads of a warp, which
  // stage rows at scattered positions, hit distinct banks
  constexpr bool kAlias = sizeof(T) == 8;
  constexpr int kSjStride = 21;
  constexpr int kSjBytes = kTileObs * kSjStride * (int)sizeof(T);
  constexpr int kS9Bytes = kTileObs * 9 * (int)sizeof(T);
  __shared__ __align__(16) unsigned char lin_smem[kAlias ? kSjBytes : kSjBytes + kS9Bytes];
  T (*sj)[kSjStride] = reinterpret_cast<T (*)[kSjStride]>(lin_smem);
  T (*s9)[9] = reinterpret_cast<T (*)[9]>(lin_smem + (kAlias ? 0 : kSjBytes));
  __shared__ uint16_t sbeg[kTileObs];
  __shared__ int srow[kTileObs];
  __shared__ double sred[kTileObs];
  // the pair table in shared memory: the lanes of a warp read different entries, which the
  // constant cache would serve one address at a time
  __shared__ uchar4 spairs[kLinVals];

  if (gate && *gate == 0) return;  // the state did not change: the linearisation is current
  if (threadIdx.x < kLinVals) spairs[threadIdx.x] = kLinPairs.v[threadIdx.x];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int L0 = tp.tile_lm0[tile], L1 = tp.tile_lm0[tile + 1];
  const int o0 = tp.lm_seg[L0], n = tp.lm_seg[L1] - o0;
  const int S0 = tp.tile_slot0[tile], ns = tp.tile_slot0[tile + 1] - S0;
  for (int i = tid; i < ns; i += blockDim.x) {
    int bg = tp.slot_beg[S0 + i], rw = tp.slot_row[S0 + i];
    POBA_CHK(tp.chk, bg, n, kChkLinSeg);
    POBA_CHK(tp.chk, rw, tp.n_slots, kChkLinRow);
    sbeg[i] = (uint16_t)bg;
    srow[i] = rw;
  }

  T jp[18], jl[6], rr[2];
  int pos = 0;
  double cost = 0.0;
  const bool active = tid < n;
  if (active) {
    const int o = o0 + tid;
    int c = tp.cam_of[o], l = tp.lm_of[o];
    POBA_CHK(tp.chk, c, tp.n_cams, kChkLinCam);
    POBA_CHK(tp.chk, l, tp.n_lms, kChkLinLm);
    pos = tp.obs_meta[o] & 0xff;
    POBA_CHK(tp.chk, pos, n, kChkLinPos);
    if (kChecks) {
      int sl = tp.obs_meta[o] >> 8;
      POBA_CHK(tp.chk, sl, ns, kChkLinSlot);
    }
    const T sw = kWeighted ? sqrt_w[o] : (T)1;
    bal_residual_jacobian<T>(prep + (size_t)c * kCamPrep, lms[l * 3 + 0], lms[l * 3 + 1],
                             lms[l * 3 + 2], obs[o], sw, jp, jl, rr);
    const size_t pad = (size_t)tp.n_obs_pad;
    store_J(J, pad, o, jp, jl);
    r[o] = rr[0];
    r[pad + o] = rr[1];
    cost = 0.5 * ((double)rr[0] * (double)rr[0] + (double)rr[1] * (double)rr[1]);
    // landmark contributions: J_l^T J_l (6 unique) and J_l^T r (3)
    s9[tid][0] = jl[0] * jl[0] + jl[3] * jl[3];
    s9[tid][1] = jl[0] * jl[1] + jl[3] * jl[4];
    s9[tid][2] = jl[0] * jl[2] + jl[3] * jl[5];
    s9[tid][3] = jl[1] * jl[1] + jl[4] * jl[4];
    s9[tid][4] = jl[1] * jl[2] + jl[4] * jl[5];
    s9[tid][5] = jl[2] * jl[2] + jl[5] * jl[5];
    s9[tid][6] = jl[0] * rr[0] + jl[3] * rr[1];
    s9[tid][7] = jl[1] * rr[0] + jl[4] * rr[1];
    s9[tid][8] = jl[2] * rr[0] + jl[5] * rr[1];
  }
  __syncthreads();
  // per-landmark sums (float32 inside the segment in FP32-bulk mode)
  if (tid < L1 - L0) {
    const int l = L0 + tid;
    const int a = tp.lm_seg[l] - o0, b = tp.lm_seg[l + 1] - o0;
    T acc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = (T)0;
    for (int q = a; q < b; ++q) {
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] += s9[q][k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) V[(size_t)l * 6 + k] = (double)acc[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) b_l[(size_t)l * 3 + k] = (double)acc[6 + k];
  }
  // J_p and r of each observation staged once at its camera-sorted position; then thread
  // (slot, entry) sums entry `entry` of the slot's J_p^T J_p / J_p^T r over the slot's rows in
  // row order (FP32-bulk: in float inside the slot segment; FP64: two FMAs per row)
  if constexpr (kAlias) __syncthreads();  // the landmark sums above have read s9
  if (active) {
#pragma unroll
    for (int e = 0; e < 18; ++e) sj[pos][e] = jp[e];
    sj[pos][18] = rr[0];
    sj[pos][19] = rr[1];
  }
  __syncthreads();
  for (int pr = tid; pr < ns * kLinVals; pr += blockDim.x) {
    const int sl = pr / kLinVals, e = pr - sl * kLinVals;
    const int beg = sbeg[sl], end = (sl + 1 < ns) ? (int)sbeg[sl + 1] : n;
    const uchar4 ix = spairs[e];
    T acc = (T)0;
    for (int q = beg; q < end; ++q) {
      if constexpr (sizeof(T) == 8)
        acc = fma(sj[q][ix.x], sj[q][ix.y], fma(sj[q][ix.z], sj[q][ix.w], acc));
      else
        acc += sj[q][ix.x] * sj[q][ix.y] + sj[q][ix.z] * sj[q][ix.w];
    }
    partial[(size_t)srow[sl] * kLinVals + e] = acc;
  }
  // block cost (fixed order)
  const double tot = block_sum_tile(cost, sred);
  if (tid == 0 && block_cost) block_cost[tile] = tot;
}

template <typename T>
void launch_linearize(const Topology& tp, const T* prep, const double* lms, const vec2<T>* obs,
                      const T* sqrt_w, T* J, T* r, double* V, double* b_l, T* partial,
                      double* block_cost, cudaStream_t s, const int32_t* gate) {
  if (sqrt_w)
    linearize_kernel<T, true><<<tp.n_tiles, kTileObs, 0, s>>>(tp, prep, lms, obs, sqrt_w, J, r, V,
                                                             b_l, partial, block_cost, gate);
  else
    linearize_kernel<T, false><<<tp.n_tiles, kTileObs, 0, s>>>(tp, prep, lms, obs, sqrt_w, J, r,
                                                              V, b_l, partial, block_cost, gate);
}
template void launch_linearize<double>(const Topology&, const double*, const double*,
                                       const double2*, const double*, double*, double*, double*,
                                       double*, double*, double*, cudaStream_t, const int32_t*);
template void launch_linearize<float>(const Topology&, const float*, const double*,
                                      const float2*, const float*, float*, float*, double*,
                                      double*, float*, double*, cudaStream_t, const int32_t*);

// ---------------------------------------------------------------------------------------
// Per camera (one block of 4 x kLinVals threads): U (45 packed) and b_p (9) summed over the
// camera's slot rows: thread (j, k) adds entry k of rows r0 + j, r0 + j + 4, ... (its row class
// j mod 4, four loads in flight at a time), thread (0, k) also the last (rows mod 4) rows, and
// the four class sums are combined as (a0 + a1) + (a2 + a3).  FP32 bulk: each thread adds its
// rows in float over runs of kLinRun rows (a segment of tiles) and the runs in double, so that
// the float-to-double conversions and double adds, which run on the FP64 pipe, are one per run
// rather than one per row.
constexpr int kLinRun = 16;
template <typename PT>
__global__ void __launch_bounds__(4 * kLinVals) lin_camera_reduce_kernel(
    Topology tp, const PT* __restrict__ partial, double* __restrict__ U45,
    double* __restrict__ b_p, const int32_t* __restrict__ gate) {
  constexpr int per = kLinVals;
  __shared__ double part[4][per];
  const int c = blockIdx.x;
  const int j = threadIdx.x / per, k = threadIdx.x - j * per;
  if (gate && *gate == 0) return;  // (block-uniform)
  // the camera's slot rows are contiguous (camera-major)
  int r0 = tp.cam_slot_ptr[c], r1 = tp.cam_slot_ptr[c + 1];
  if (kChecks && (r0 < 0 || r1 < r0 || r1 > tp.n_slots)) {
    int bad = r1 > tp.n_slots ? r1 : r0;
    POBA_CHK(tp.chk, bad, 0, kChkCamReduce);
    r0 = r1 = 0;
  }
  const int rm = r0 + ((r1 - r0) & ~3);  // end of the rows shared round-robin
  double a = 0.0;
  int r = r0 + j;
  if constexpr (sizeof(PT) == 4) {
    // runs of kLinRun of this thread's rows in float, the runs in double
    while (r < rm) {
      float f = 0.f;
      const int re = min(rm, r + 4 * kLinRun);
      for (; r + 12 < re; r += 16) {
        const float v0 = __ldcg(partial + (size_t)r * per + k);
        const float v1 = __ldcg(partial + (size_t)(r + 4) * per + k);
        const float v2 = __ldcg(partial + (size_t)(r + 8) * per + k);
        const float v3 = __ldcg(partial + (size_t)(r + 12) * per + k);
        f += v0;
        f += v1;
        f += v2;
        f += v3;
      }
      for (; r < re; r += 4) f += __ldcg(partial + (size_t)r * per + k);
      a += (double)f;
    }
    if (j == 0) {
      float f = 0.f;
      for (r = rm; r < r1; ++r) f += __ldcg(partial + (size_t)r * per + k);
      a += (double)f;
    }
  } else {
    for (; r + 12 < rm; r += 16) {
      const PT v0 = __ldcg(partial + (size_t)r * per + k);
      const PT v1 = __ldcg(partial + (size_t)(r + 4) * per + k);
      const PT v2 = __ldcg(partial + (size_t)(r + 8) * per + k);
      const PT v3 = __ldcg(partial + (size_t)(r + 12) * per + k);
      a += (double)v0;
      a += (double)v1;
      a += (double)v2;
      a += (double)v3;
    }
    for (; r < rm; r += 4) a += (double)__ldcg(partial + (size_t)r * per + k);
    if (j == 0)
      for (r = rm; r < r1; ++r) a += (double)__ldcg(partial + (size_t)r * per + k);
  }
  part[j][k] = a;
  __syncthreads();
  if (j == 0) {
    const double acc = (part[0][k] + part[1][k]) + (part[2][k] + part[3][k]);
    if (k < 45) U45[(size_t)c * 45 + k] = acc;
    else b_p[(size_t)c * 9 + (k - 45)] = acc;
  }
}

template <typename PT>
void launch_lin_camera_reduce(const Topology& tp, const PT* partial, double* U45, double* b_p,
                              cudaStream_t s, const int32_t* gate) {
  lin_camera_reduce_kernel<PT><<<tp.n_cams, 4 * kLinVals, 0, s>>>(tp, partial, U45, b_p, gate);
}
// Long tracks: the linearisation kernel leaves each piece's own sums in V and b_l; the track's
// V = sum J_l^T J_l and b_l = sum J_l^T r are the sums over its pieces, added in piece order (in
// double) and written back to every piece.  One thread per long track.
__global__ void long_track_blocks_kernel(Topology tp, double* __restrict__ V,
                                         double* __restrict__ b_l,
                                         const int32_t* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= tp.n_long) return;
  const int l0 = tp.long_first[j], np = tp.long_np[j];
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  for (int q = 0; q < np; ++q) {
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += V[(size_t)(l0 + q) * 6 + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[6 + k] += b_l[(size_t)(l0 + q) * 3 + k];
  }
  for (int q = 0; q < np; ++q) {
#pragma unroll
    for (int k = 0; k < 6; ++k) V[(size_t)(l0 + q) * 6 + k] = acc[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) b_l[(size_t)(l0 + q) * 3 + k] = acc[6 + k];
  }
}

void launch_long_track_blocks(const Topology& tp, double* V, double* b_l, cudaStream_t s,
                              const int32_t* gate) {
  if (tp.n_long <= 0) return;
  long_track_blocks_kernel<<<(tp.n_long + 127) / 128, 128, 0, s>>>(tp, V, b_l, gate);
}

template void launch_lin_camera_reduce<double>(const Topology&, const double*, double*, double*, cudaStream_t, const int32_t*);
template void launch_lin_camera_reduce<float>(const Topology&, const float*, double*, double*, cudaStream_t, const int32_t*);

// ---------------------------------------------------------------------------------------
// Damping (reading of D: D^T D = diag(J^T J) clamped to [1e-6, 1e32], or D = I) and block
// Cholesky inverses A^-1 = L^-T L^-1 in float64.  Blocks [0, cam_blocks) handle cameras, the
// rest landmarks.

// Camera blocks: kCamBlock cameras x 9 threads.  Thread k of a camera loads row k; the 9
// threads factor A = L L^T column by column (the diagonal keeps 1/L_jj, from rsqrt); thread k
// then computes column k of M = L^-1 by forward substitution and row k of A^-1 = M^T M.
// Landmark blocks: one thread per landmark, the same steps for a 3x3 block.
constexpr int kDampThreads = kCamBlock * 9;

__global__ void __launch_bounds__(kDampThreads) damp_invert_kernel(
    Topology tp, const double* __restrict__ U45, const double* __restrict__ V,
    const double* __restrict__ lambda, int lam_stride, int mode, int cam_blocks,
    double* __restrict__ Uinv, double* __restrict__ Vinv, float* __restrict__ Vinv_f,
    int32_t* __restrict__ not_spd) {
  const int tid = threadIdx.x;
  if ((int)blockIdx.x < cam_blocks) {
    __shared__ double A[kCamBlock][9][10];
    __shared__ double M[kCamBlock][9][10];
    const int cl = tid / 9, k = tid - cl * 9;
    const int c = blockIdx.x * kCamBlock + cl;
    const bool ok_cam = c < tp.n_cams;
    if (ok_cam) {
      const double lam = lambda[(size_t)tp.cam_prob[c] * lam_stride];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const int i0 = k < j ? k : j, j0 = k < j ? j : k;
        A[cl][k][j] = U45[(size_t)c * 45 + packed9(i0, j0)];
      }
      A[cl][k][k] += damp_diag(A[cl][k][k], lam, mode);
    }
    __syncthreads();
    // left-looking Cholesky, one column per step: threads k >= j update row k of column j
    // in parallel; thread j then takes the reciprocal square root of the pivot.
    __shared__ int bad[kCamBlock];
    if (k == 0) bad[cl] = 0;
    for (int j = 0; j < 9; ++j) {
      if (ok_cam && k >= j) {
        double v = A[cl][k][j];
        for (int p = 0; p < j; ++p) v -= A[cl][k][p] * A[cl][j][p];
        A[cl][k][j] = v;
      }
      __syncthreads();
      if (ok_cam && k == j) {
        double d = A[cl][j][j];
        if (!(d > 0.0) || !isfinite(d)) {
          bad[cl] = 1;
          d = 1.0;
        }
        A[cl][j][j] = rsqrt(d);  // 1 / L_jj
      }
      __syncthreads();
      if (ok_cam && k > j) A[cl][k][j] *= A[cl][j][j];
      __syncthreads();
    }
    if (ok_cam && k == 0 && bad[cl]) atomicOr(not_spd + tp.cam_prob[c], 1);
    if (ok_cam) {
      const double (*a)[10] = A[cl];
      double m[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) m[i] = 0.0;
      m[k] = a[k][k];
      for (int i = k + 1; i < 9; ++i) {
        double v = 0.0;
        for (int p = k; p < i; ++p) v -= a[i][p] * m[p];
        m[i] = v * a[i][i];
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) M[cl][i][k] = m[i];
    }
    __syncthreads();
    if (ok_cam) {
      double* out = Uinv + (size_t)c * 81 + k * 9;
      for (int j = 0; j < 9; ++j) {
        double v = 0.0;
        for (int p = (k > j ? k : j); p < 9; ++p) v += M[cl][p][k] * M[cl][p][j];
        out[j] = v;
      }
    }
  } else {
    const int l = (blockIdx.x - cam_blocks) * blockDim.x + tid;
    if (l >= tp.n_lms) return;
    const double lam = lambda[(size_t)tp.lm_prob[l] * lam_stride];
    const double* v = V + (size_t)l * 6;
    const double a00 = v[0] + damp_diag(v[0], lam, mode), a01 = v[1], a02 = v[2];
    const double a11 = v[3] + damp_diag(v[3], lam, mode), a12 = v[4];
    const double a22 = v[5] + damp_diag(v[5], lam, mode);
    bool ok = true;
    double d0 = a00;
    if (!(d0 > 0.0) || !isfinite(d0)) { ok = false; d0 = 1.0; }
    const double m00 = rsqrt(d0);  // 1 / l00
    const double l10 = a01 * m00, l20 = a02 * m00;
    double d1 = a11 - l10 * l10;
    if (!(d1 > 0.0) || !isfinite(d1)) { ok = false; d1 = 1.0; }
    const double m11 = rsqrt(d1);
    const double l21 = (a12 - l20 * l10) * m11;
    double d2 = a22 - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0) || !isfinite(d2)) { ok = false; d2 = 1.0; }
    const double m22 = rsqrt(d2);
    if (!ok) atomicOr(not_spd + tp.lm_prob[l], 1);
    // M = L^-1
    const double m10 = -l10 * m00 * m11;
    const double m21 = -l21 * m11 * m22;
    const double m20 = -(l20 * m00 + l21 * m10) * m22;
    // Vinv = M^T M, 6 unique entries [00 01 02 11 12 22]
    double o[6];
    o[0] = m00 * m00 + m10 * m10 + m20 * m20;
    o[1] = m10 * m11 + m20 * m21;
    o[2] = m20 * m22;
    o[3] = m11 * m11 + m21 * m21;
    o[4] = m21 * m22;
    o[5] = m22 * m22;
#pragma unroll
    for (int q = 0; q < 6; ++q) Vinv[(size_t)l * 6 + q] = o[q];
    if (Vinv_f) {
#pragma unroll
      for (int q = 0; q < 6; ++q) Vinv_f[(size_t)l * 6 + q] = (float)o[q];
    }
  }
}

void launch_damp_invert(const Topology& tp, const double* U45, const double* V,
                        const double* lambda, int lam_stride, int damping_mode, double* Uinv,
                        double* Vinv, float* Vinv_f, int32_t* not_spd, cudaStream_t s) {
  const int cb = (tp.n_cams + kCamBlock - 1) / kCamBlock;
  const int lb = (tp.n_lms + kDampThreads - 1) / kDampThreads;
  damp_invert_kernel<<<cb + lb, kDampThreads, 0, s>>>(tp, U45, V, lambda, lam_stride, damping_mode,
                                                     cb, Uinv, Vinv, Vinv_f, not_spd);
}

// Cameras only: out81[c] = (A45[c] + damping at lambda)^-1 (the same factorisation as above).
void launch_invert_camera_blocks(const Topology& tp, const double* A45, const double* lambda,
                                 int damping_mode, double* out81, int32_t* not_spd,
                                 cudaStream_t s) {
  const int cb = (tp.n_cams + kCamBlock - 1) / kCamBlock;
  damp_invert_kernel<<<cb, kDampThreads, 0, s>>>(tp, A45, nullptr, lambda, 0, damping_mode, cb,
                                                 out81, nullptr, nullptr, not_spd);
}

// ---------------------------------------------------------------------------------------
// Cost in float64 at (cameras prepared in `prep`, landmarks lms + dx_l): one block per tile,
// tile_cost[t] = sum over the tile's observations of w ||r||^2 (fixed order).
__global__ void __launch_bounds__(kTileObs) tile_cost_kernel(
    Topology tp, const double* __restrict__ prep, const double* __restrict__ lms,
    const double* __restrict__ dx_l, const double2* __restrict__ obs,
    const double* __restrict__ sqrt_w, double* __restrict__ tile_cost) {
  __shared__ double sred[kTileObs];
  const int4 d = tp.tile_desc[2 * blockIdx.x];
  const int o0 = d.z, n = d.w;
  double e = 0.0;
  if ((int)threadIdx.x < n) {
    const int o = o0 + threadIdx.x;
    int c = tp.cam_of[o], l = tp.lm_of[o];
    POBA_CHK(tp.chk, c, tp.n_cams, kChkCostCam);
    POBA_CHK(tp.chk, l, tp.n_lms, kChkCostLm);
    const double* q = prep + (size_t)c * kCamPrep;
    double X0 = lms[l * 3 + 0], X1 = lms[l * 3 + 1], X2 = lms[l * 3 + 2];
    if (dx_l) {
      X0 += dx_l[l * 3 + 0];
      X1 += dx_l[l * 3 + 1];
      X2 += dx_l[l * 3 + 2];
    }
    const double P0 = q[0] * X0 + q[1] * X1 + q[2] * X2 + q[18];
    const double P1 = q[3] * X0 + q[4] * X1 + q[5] * X2 + q[19];
    const double P2 = q[6] * X0 + q[7] * X1 + q[8] * X2 + q[20];
    const double iz = 1.0 / P2;
    const double px = -P0 * iz, py = -P1 * iz;
    const double n2 = px * px + py * py;
    const double rad = 1.0 + n2 * (q[22] + q[23] * n2);
    const double2 ob = obs[o];
    const double r0 = q[21] * rad * px - ob.x, r1 = q[21] * rad * py - ob.y;
    e = r0 * r0 + r1 * r1;
    if (sqrt_w) e *= sqrt_w[o] * sqrt_w[o];
  }
  const double tot = block_sum_tile(e, sred);
  if (threadIdx.x == 0) tile_cost[blockIdx.x] = tot;
}

void launch_tile_cost(const Topology& tp, const double* prep, const double* lms,
                      const double* dx_l, const double2* obs, const double* sqrt_w,
                      double* tile_cost, cudaStream_t s) {
  tile_cost_kernel<<<tp.n_tiles, kTileObs, 0, s>>>(tp, prep, lms, dx_l, obs, sqrt_w, tile_cost);
}

}  // namespace poba
