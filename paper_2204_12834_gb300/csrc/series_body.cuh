// Device bodies of one power-series term (Sec. 4.3), shared by the per-term kernels and the
// persistent series kernel.  Data written by other blocks of the same launch (t_cam, partial,
// x) is read with __ldcg (L2), since L1 is not coherent across SMs within a launch.
//
// With P = U^-1 W V^-1 W^T, W = J_p^T J_l, a term t_i = P t_{i-1} is applied matrix-free:
//   tile body (per tile of whole landmarks, one observation per thread):
//     u_o = J_p,o t_c(o)                       (t staged per slot in shared memory)
//     z_l = V_l^-1 sum_{o in l} J_l,o^T u_o    (landmark-segmented sum in shared memory)
//     g_o = J_p,o^T (J_l,o z_l(o))             (J still in registers: one J read per term)
//     partial[row(slot)] = sum_{o in slot} g_o (per-tile camera sums, fixed order)
//   camera body (9 threads per camera):
//     y_c = sum of the camera's partial rows; t_i = U_c^-1 y_c; x += t_i; t_cam[c] = t_i.
// With z_l = V_l^-1 b_l (RHS mode) the same bodies form b~ = b_p - W V^-1 b_l and
// x(0) = -U^-1 b~ (Sec. 4.2 and eq. `x_approx` with m = 0).
#pragma once

#include <cstddef>
#include <cstdint>

#include "poba_internal.cuh"
#include "tile_common.cuh"

namespace poba {

enum { kModeSeries = 0, kModeRhs = 1 };

// FP32 tiles whose slots hold fewer rows than this on average sum each (slot, component) in one
// thread; longer slots are split over a warp.
constexpr int kShortSlotRows = 6;

template <typename T>
__device__ __forceinline__ void load_J(const T* __restrict__ J, size_t pad, int o, T (&jp)[18],
                                       T (&jl)[6]) {
#pragma unroll
  for (int p = 0; p < 18; ++p) jp[p] = J[p * pad + o];
#pragma unroll
  for (int p = 0; p < 6; ++p) jl[p] = J[(18 + p) * pad + o];
}

// z = Vinv s with Vinv stored as [00 01 02 11 12 22].
template <typename T>
__device__ __forceinline__ void apply_vinv(const T* __restrict__ vi, const T (&s)[3], T (&z)[3]) {
  const T v0 = vi[0], v1 = vi[1], v2 = vi[2], v3 = vi[3], v4 = vi[4], v5 = vi[5];
  z[0] = v0 * s[0] + v1 * s[1] + v2 * s[2];
  z[1] = v1 * s[0] + v3 * s[1] + v4 * s[2];
  z[2] = v2 * s[0] + v4 * s[1] + v5 * s[2];
}

// Tile header: {L0, nl, o0, n} and {S0, ns}.
struct TileHdr {
  int L0, nl, o0, n, S0, ns;
};

__device__ __forceinline__ TileHdr load_tile(const Topology& tp, int tile) {
  const int4 a = tp.tile_desc[2 * tile], b = tp.tile_desc[2 * tile + 1];
  return TileHdr{a.x, a.y, a.z, a.w, b.x, b.y};
}

// 16-byte aligned: the persistent kernel reuses sg as a double array in its camera phase.
template <typename T>
struct __align__(16) TileSmem {
  T tcam[kTileObs][9];
  T sv[kTileObs][3];
  T sg[kTileObs][9];
  uint16_t sbeg[kTileObs];
  int srow[kTileObs];
  int sseg[kTileLms + 1];
};
static_assert(offsetof(TileSmem<float>, sg) % 8 == 0, "sg is reused as double storage");
static_assert(offsetof(TileSmem<double>, sg) % 8 == 0, "sg is reused as double storage");

// One tile of one term (blockDim.x == kTileObs; every thread must call it).
template <typename T, int MODE>
__device__ __forceinline__ void tile_matvec_body(const Topology& tp, int tile,
                                                 const T* __restrict__ J,
                                                 const T* __restrict__ t_cam,
                                                 const double* __restrict__ b_l,
                                                 const T* __restrict__ Vinv,
                                                 T* __restrict__ partial, TileSmem<T>& sm) {
  const int tid = threadIdx.x;
  const TileHdr th = load_tile(tp, tile);
  const int o0 = th.o0, n = th.n, ns = th.ns, nl = th.nl;
  const bool active = tid < n;
  const size_t pad = (size_t)tp.n_obs_pad;
  // issue every independent load of the tile before the first barrier
  T jp[18], jl[6];
  int meta = 0;
  if (active) {
    const int o = o0 + tid;
    meta = tp.obs_meta[o];
    load_J(J, pad, o, jp, jl);
  }
  T vi[6];
  double bl[3] = {0.0, 0.0, 0.0};
  if (tid < nl) {
#pragma unroll
    for (int k = 0; k < 6; ++k) vi[k] = Vinv[(size_t)(th.L0 + tid) * 6 + k];
    if (MODE == kModeRhs) {
#pragma unroll
      for (int k = 0; k < 3; ++k) bl[k] = b_l[(size_t)(th.L0 + tid) * 3 + k];
    }
  }
  for (int i = tid; i < ns; i += blockDim.x) {
    sm.sbeg[i] = tp.slot_beg[th.S0 + i];
    sm.srow[i] = tp.slot_row[th.S0 + i];
  }
  for (int i = tid; i <= nl; i += blockDim.x) sm.sseg[i] = tp.lm_seg[th.L0 + i] - o0;
  __syncthreads();
  if (MODE == kModeSeries) {
    // the current term of each slot's camera
    for (int i = tid; i < ns * 9; i += blockDim.x) {
      const int s = i / 9, k = i - s * 9;
      sm.tcam[s][k] = __ldcg(t_cam + (size_t)tp.slot_cam[th.S0 + s] * kTStride + k);
    }
  }
  __syncthreads();

  if (MODE == kModeSeries && active) {
    const T* tc = sm.tcam[meta >> 8];
    T u0 = (T)0, u1 = (T)0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      u0 += jp[j] * tc[j];
      u1 += jp[9 + j] * tc[j];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sm.sv[tid][k] = jl[k] * u0 + jl[3 + k] * u1;
  }
  __syncthreads();
  // landmark phase: z_l = V_l^-1 (sum of W^T t contributions, or b_l), written back per obs
  if (tid < nl) {
    const int a = sm.sseg[tid], b = sm.sseg[tid + 1];
    T s3[3];
    if (MODE == kModeSeries) {
      s3[0] = s3[1] = s3[2] = (T)0;
      for (int q = a; q < b; ++q) {
        s3[0] += sm.sv[q][0];
        s3[1] += sm.sv[q][1];
        s3[2] += sm.sv[q][2];
      }
    } else {
      s3[0] = (T)bl[0];
      s3[1] = (T)bl[1];
      s3[2] = (T)bl[2];
    }
    T z[3];
    z[0] = vi[0] * s3[0] + vi[1] * s3[1] + vi[2] * s3[2];
    z[1] = vi[1] * s3[0] + vi[3] * s3[1] + vi[4] * s3[2];
    z[2] = vi[2] * s3[0] + vi[4] * s3[1] + vi[5] * s3[2];
    for (int q = a; q < b; ++q) {
      sm.sv[q][0] = z[0];
      sm.sv[q][1] = z[1];
      sm.sv[q][2] = z[2];
    }
  }
  __syncthreads();
  // W z scatter: g_o = J_p^T (J_l z), staged at the camera-sorted position
  if (active) {
    const T z0 = sm.sv[tid][0], z1 = sm.sv[tid][1], z2 = sm.sv[tid][2];
    const T w0 = jl[0] * z0 + jl[1] * z1 + jl[2] * z2;
    const T w1 = jl[3] * z0 + jl[4] * z1 + jl[5] * z2;
    T* g = sm.sg[meta & 0xff];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = jp[j] * w0 + jp[9 + j] * w1;
  }
  __syncthreads();
  slot_sums<T, T>(sm.sg, ns, n, sm.sbeg, sm.srow, partial, 9);
}

// Phases 1-3 of the FP32-bulk tile (below), shared by the per-term tile kernel and the
// pipelined persistent kernel so that both compute the same sums in the same order.  The caller
// stages: tcam[slot * tstride .. + 9) = current term of the slot's camera; V^-1 of tile landmark l at
// vinv[l * vstride .. + 6) (RHS mode: b_l at + 6 .. + 9); sseg[l] = tile-relative segment
// offsets (nl + 1 entries); sbeg[s] = first camera-sorted position of slot s; srow[s] = its
// camera-major row.  lm = the observation's landmark within the tile, meta = pos | slot << 8.
// kShared: the caller's staging shares storage (landmark marks in sv, V^-1 in sg), which costs
// two more barriers; otherwise sv, sg, tcam and vinv must be separate.  hook() runs after the
// barrier that follows the v writes (every thread has passed the start of the tile).  Every
// thread of the block must call it.
template <int MODE, bool kShared, typename SegT, typename BegT, typename Hook>
__device__ __forceinline__ void f32_tile_core(bool active, int n, int ns, int lm, int meta,
                                              const float (&jp)[18], const float (&jl)[6],
                                              const float* tcam, int tstride, const float* vinv,
                                              int vstride, const SegT* sseg, const BegT* sbeg,
                                              const int* srow, float (*sv)[3], float (*sg)[9],
                                              float* __restrict__ partial, Hook&& hook) {
  const int tid = threadIdx.x;
  // phase 1: u = J_p t, v = J_l^T u
  float u0 = 0.f, u1 = 0.f;
  if (MODE == kModeSeries && active) {
    const float* tc = tcam + (size_t)(meta >> 8) * tstride;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      u0 += jp[j] * tc[j];
      u1 += jp[9 + j] * tc[j];
    }
  }
  if (kShared) __syncthreads();  // sv still holds the landmark marks read before the call
  if (MODE == kModeSeries && active) {
#pragma unroll
    for (int k = 0; k < 3; ++k) sv[tid][k] = jl[k] * u0 + jl[3 + k] * u1;
  }
  __syncthreads();
  hook();
  // phase 2: each observation thread sums its landmark's v in segment order, applies V^-1 and
  // forms J_l z
  if (active) {
    float s3[3];
    const float* vl = vinv + (size_t)lm * vstride;
    if (MODE == kModeSeries) {
      s3[0] = s3[1] = s3[2] = 0.f;
      const int a = sseg[lm], b = sseg[lm + 1];
      for (int q = a; q < b; ++q) {
        s3[0] += sv[q][0];
        s3[1] += sv[q][1];
        s3[2] += sv[q][2];
      }
    } else {
      s3[0] = vl[6];
      s3[1] = vl[7];
      s3[2] = vl[8];
    }
    const float z0 = vl[0] * s3[0] + vl[1] * s3[1] + vl[2] * s3[2];
    const float z1 = vl[1] * s3[0] + vl[3] * s3[1] + vl[4] * s3[2];
    const float z2 = vl[2] * s3[0] + vl[4] * s3[1] + vl[5] * s3[2];
    u0 = jl[0] * z0 + jl[1] * z1 + jl[2] * z2;
    u1 = jl[3] * z0 + jl[4] * z1 + jl[5] * z2;
  }
  if (kShared) __syncthreads();  // the V^-1 staging shares sg with the scatter below
  if (active) {
    float* g = sg[meta & 0xff];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = jp[j] * u0 + jp[9 + j] * u1;
  }
  __syncthreads();
  // phase 3, chosen by the tile's shape (the same choice in every form):
  //  * short slots (fewer than kShortSlotRows rows on average): one thread per (slot, component)
  //    sums the slot's rows in row order;
  //  * otherwise one warp per slot: lane 3 k + c sums component k over the c-th third of the
  //    slot's rows in row order, and the three thirds are added in chunk order.
  if (n < kShortSlotRows * ns) {
    for (int k = tid; k < ns * 9; k += blockDim.x) {
      const int sl = k / 9, kc = k - 9 * sl;
      const int beg = sbeg[sl], end = (sl + 1 < ns) ? (int)sbeg[sl + 1] : n;
      float acc = 0.f;
      for (int q = beg; q < end; ++q) acc += sg[q][kc];
      partial[(size_t)srow[sl] * 9 + kc] = acc;
    }
    return;
  }
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  const int kc = lane / 3, cc = lane - 3 * kc;
  for (int sl = warp; sl < ns; sl += nw) {
    const int beg = sbeg[sl], end = (sl + 1 < ns) ? (int)sbeg[sl + 1] : n;
    const int chunk = (end - beg + 2) / 3;
    float acc = 0.f;
    if (lane < 27) {
      const int q0 = beg + cc * chunk, q1 = min(q0 + chunk, end);
      for (int q = q0; q < q1; ++q) acc += sg[q][kc];
    }
    const float a1 = __shfl_down_sync(0xffffffffu, acc, 1);
    const float a2 = __shfl_down_sync(0xffffffffu, acc, 2);
    if (lane < 27 && cc == 0) partial[(size_t)srow[sl] * 9 + kc] = (acc + a1) + a2;
  }
}

// FP32-bulk tile body (blockDim.x == kTileObs; every thread must call it).  The same sums as
// tile_matvec_body, arranged for float arithmetic, where redundant FMAs are cheap and barriers
// are not:
//   phase 0  J and the observation code into registers; slot threads stage their slot's
//            first position, camera-major row and current term row; landmark threads stage
//            their segment, V^-1 and (RHS) b_l and mark their observations' landmark;
//   phase 1  u = J_p t, v = J_l^T u per observation;
//   phase 2  every observation thread sums its own landmark's v in segment order and applies
//            V^-1 (the same sum and the same z in every thread of the landmark), then scatters
//            g = J_p^T (J_l z) to its camera-sorted position;
//   phase 3  tiles of short slots: one thread per (slot, component) sums the slot's rows in
//            order; otherwise one warp per slot: 27 lanes, one per (component, third of the
//            slot's rows), sum their rows in order, the thirds are added in order; either way
//            the sum is written to the slot's camera-major row.
template <int MODE>
__device__ __forceinline__ void tile_matvec_body_f32(const Topology& tp, int tile,
                                                     const float* __restrict__ J,
                                                     const float* __restrict__ t_cam,
                                                     const double* __restrict__ b_l,
                                                     const float* __restrict__ Vinv,
                                                     float* __restrict__ partial,
                                                     TileSmem<float>& sm) {
  const int tid = threadIdx.x;
  const TileHdr th = load_tile(tp, tile);
  const int o0 = th.o0, n = th.n, ns = th.ns, nl = th.nl;
  const bool active = tid < n;
  const size_t pad = (size_t)tp.n_obs_pad;
  float jp[18], jl[6];
  int meta = 0;
  if (active) {
    const int o = o0 + tid;
    meta = tp.obs_meta[o];
    load_J(J, pad, o, jp, jl);
  }
  // shared arrays reused here: sbeg / srow per slot, sseg per landmark, tcam per slot,
  // sv per observation (first the landmark index of each observation, then v);
  // sg[l][0..5] = V^-1 of landmark l and sg[l][6..8] = b_l (RHS) until phase 2 ends
  for (int i = tid; i < ns; i += blockDim.x) {
    const int r = tp.slot_row[th.S0 + i];
    sm.sbeg[i] = tp.slot_beg[th.S0 + i];
    sm.srow[i] = r;
    if (MODE == kModeSeries) {
      const int c = tp.slot_cam[th.S0 + i];
#pragma unroll
      for (int k = 0; k < 9; ++k) sm.tcam[i][k] = __ldcg(t_cam + (size_t)c * kTStride + k);
    }
  }
  if (tid < nl) {
    const int a = tp.lm_seg[th.L0 + tid] - o0, b = tp.lm_seg[th.L0 + tid + 1] - o0;
    sm.sseg[tid] = a;
    if (tid == nl - 1) sm.sseg[nl] = b;
#pragma unroll
    for (int k = 0; k < 6; ++k) sm.sg[tid][k] = Vinv[(size_t)(th.L0 + tid) * 6 + k];
    if (MODE == kModeRhs) {
#pragma unroll
      for (int k = 0; k < 3; ++k) sm.sg[tid][6 + k] = (float)b_l[(size_t)(th.L0 + tid) * 3 + k];
    }
    for (int q = a; q < b; ++q) sm.sv[q][0] = __int_as_float(tid);  // landmark of each obs
  }
  __syncthreads();
  const int lm = active ? __float_as_int(sm.sv[tid][0]) : 0;
  f32_tile_core<MODE, true>(active, n, ns, lm, meta, jp, jl, &sm.tcam[0][0], 9, &sm.sg[0][0], 9,
                            sm.sseg, sm.sbeg, sm.srow, sm.sv, sm.sg, partial, [] {});
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}

// Sum of one chunk of a camera's slot rows, component k: rows [q0, q1) in row order (loads are
// issued 16 floats or 8 doubles at a time).  A chunk is a segment: FP32-bulk rows are added in
// float inside it and the chunks in double (camera_body), FP64 rows in double throughout.
template <typename PT>
__device__ __forceinline__ double cam_chunk_sum(const PT* __restrict__ partial, int q0, int q1,
                                                int k) {
  constexpr int B = sizeof(PT) == 4 ? 16 : 8;
  PT pc = (PT)0;
  for (int rb = q0; rb < q1; rb += B) {
    PT buf[B];
#pragma unroll
    for (int j = 0; j < B; ++j)
      buf[j] = (rb + j < q1) ? __ldcg(partial + (size_t)(rb + j) * 9 + k) : (PT)0;
#pragma unroll
    for (int j = 0; j < B; ++j) pc += buf[j];
  }
  return (double)pc;
}

// Camera body for cameras [cam0, cam0 + per_block): thread (c, k) sums component k of the
// camera's contiguous slot rows (chunk by chunk, cam_chunk_rows rows per chunk, the chunks in
// order), applies row k of U^-1, updates x and writes the new term t_cam[c]; then the 9 threads
// of the camera add their squared term and x components (in component order) into the camera's
// pair cam_norm[c] = (||t_c||^2, ||x_c||^2).  Cameras of problems whose series has stopped are
// left as they are.  FP64 work is one add per slot row and component: every FP64 warp
// instruction costs 16 pipe cycles on GB300, so no shuffle trees are used for the slot sums.
// ys and y2 are shared [per_block][9] arrays.  Every thread of the block must call it.
template <typename PT, int MODE>
__device__ __forceinline__ void camera_body(const Topology& tp, int cam0, int per_block,
                                            const PT* __restrict__ partial,
                                            const double* __restrict__ b_p,
                                            const double* __restrict__ Uinv,
                                            double* __restrict__ x, PT* __restrict__ t_cam,
                                            const SeriesState* st, double* __restrict__ cam_norm,
                                            double (*ys)[9], double (*y2)[9]) {
  const int tid = threadIdx.x;
  const int cl = tid / 9, k = tid - cl * 9;
  const int c = cam0 + cl;
  const bool cam_ok = cl < per_block && c < tp.n_cams && !ld_volatile(&st[tp.cam_prob[c]].done);
  double y = 0.0;
  if (cam_ok) {
    const int r0 = tp.cam_slot_ptr[c], r1 = tp.cam_slot_ptr[c + 1];
    const int C = cam_chunk_rows(r1 - r0);
    for (int q0 = r0; q0 < r1; q0 += C) y += cam_chunk_sum(partial, q0, min(q0 + C, r1), k);
  }
  if (MODE == kModeRhs && cam_ok) y = b_p[(size_t)c * 9 + k] - y;  // b~ = b_p - W V^-1 b_l
  if (cl < per_block) ys[cl][k] = y;
  __syncthreads();
  double v = 0.0, xv = 0.0;
  if (cam_ok) {
    const double* ui = Uinv + (size_t)c * 81 + k * 9;
#pragma unroll
    for (int j = 0; j < 9; ++j) v += ui[j] * ys[cl][j];
    if (MODE == kModeRhs) {
      v = -v;  // x(0) = -U^-1 b~
      xv = v;
    } else {
      xv = __ldcg(x + (size_t)c * 9 + k) + v;
    }
    x[(size_t)c * 9 + k] = xv;
    t_cam[(size_t)c * kTStride + k] = (PT)v;
  }
  __syncthreads();
  if (cl < per_block) {
    ys[cl][k] = v * v;
    y2[cl][k] = xv * xv;
  }
  __syncthreads();
  if (cam_ok && k == 0) {
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      a += ys[cl][j];
      b += y2[cl][j];
    }
    cam_norm[2 * c + 0] = a;
    cam_norm[2 * c + 1] = b;
  }
  __syncthreads();
}

// The stop rule of eq. `qcriterion` at term `iter` from the squared norms; updates one
// problem's state.
__device__ __forceinline__ void series_stop_rule(SeriesState* st, int iter, double T2, double X2,
                                                 double eps) {
  const double tn = sqrt(T2), xn = sqrt(X2);
  st->t_norm = tn;
  st->x_norm = xn;
  st->m = iter;
  if (iter == 0) {
    st->stop_value = INFINITY;
    if (xn == 0.0) {
      st->done = 1;
      st->stopped = 1;
    }
  } else if (xn == 0.0) {
    st->stop_value = 0.0;
    st->done = 1;
    st->stopped = 1;
  } else {
    const double sv = (double)(iter + 1) * tn / xn;
    st->stop_value = sv;
    if (sv < eps) {
      st->done = 1;
      st->stopped = 1;
    }
  }
}

// Every problem still running: sum its cameras' norm pairs (one warp per problem, lanes strided
// over the cameras, then a fixed shuffle tree) and apply its stop rule for term `iter`; raise
// all_done when no problem is left.  Every thread of one block (at least one full warp) must
// call it.
__device__ __forceinline__ void problems_stop_rule(const Topology& tp,
                                                   const double* __restrict__ cam_norm,
                                                   SeriesState* st, SeriesGlobal* sgl, int iter,
                                                   double eps, int* s_running) {
  // only full warps take problems (the shuffles below use every lane of a warp)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *s_running = 0;
  __syncthreads();
  for (int p = warp; warp < nw && p < tp.n_probs; p += nw) {
    if (ld_volatile(&st[p].done)) continue;  // warp-uniform
    // lane j adds the pairs of cameras j, j + 32, j + 64, ... in that order; the loads go out
    // eight at a time so that the sum waits for one round trip per eight cameras
    double a = 0.0, b = 0.0;
    const int c1 = tp.cam_off[p + 1];
    const double2* cn = reinterpret_cast<const double2*>(cam_norm);
    for (int cb = tp.cam_off[p] + lane; cb < c1; cb += 32 * 8) {
      double2 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = cb + 32 * j < c1 ? __ldcg(cn + cb + 32 * j) : make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        a += v[j].x;
        b += v[j].y;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, off);
      b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
      series_stop_rule(&st[p], iter, a, b, eps);
      if (!st[p].done) atomicAdd(s_running, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (*s_running == 0) sgl->all_done = 1;
  }
  __syncthreads();
}

}  // namespace poba
