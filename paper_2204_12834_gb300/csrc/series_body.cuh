// Device bodies of one power-series term (Sec. 4.3), shared by the per-term kernels and the
// persistent series kernel.  Data written by other blocks of the same launch (t_cam, partial,
// x) is read with __ldcg (L2), since L1 is not coherent across SMs within a launch.
//
// With P = U^-1 W V^-1 W^T, W = J_p^T J_l, a term t_i = P t_{i-1} is applied matrix-free over
// the series schedule (SerSchedule): a block runs one group of consecutive landmarks, chunk by
// chunk (one observation per thread):
//     u_o = J_p,o t_c(o)                       (t staged per group slot in shared memory)
//     z_l = V_l^-1 sum_{o in l} J_l,o^T u_o    (landmark-segmented sum)
//     g_o = J_p,o^T (J_l,o z_l(o))             (J still in registers: one J read per term)
//     acc[slot(o)] += sum_{o in slot} g_o      (per chunk slot, then across the group's chunks)
//   and writes one partial row per group slot; then the camera body (9 threads per camera):
//     y_c = sum of the camera's partial rows; t_i = U_c^-1 y_c; x += t_i; t_cam[c] = t_i.
// With z_l = V_l^-1 b_l (RHS mode) the same bodies form b~ = b_p - W V^-1 b_l and
// x(0) = -U^-1 b~ (Sec. 4.2 and eq. `x_approx` with m = 0).
//
// Every sum has a fixed order that depends only on the schedule, whichever block runs a group,
// so all execution forms give bitwise-equal results.
#pragma once

#include <cstddef>
#include <cstdint>

#include "jacobian_io.cuh"
#include "poba_internal.cuh"
#include "tile_common.cuh"

namespace poba {

enum { kModeSeries = 0, kModeRhs = 1 };

constexpr unsigned kFull = 0xffffffffu;

// z = Vinv s with Vinv stored as [00 01 02 11 12 22].
template <typename T>
__device__ __forceinline__ void apply_vinv(const T* __restrict__ vi, const T (&s)[3], T (&z)[3]) {
  const T v0 = vi[0], v1 = vi[1], v2 = vi[2], v3 = vi[3], v4 = vi[4], v5 = vi[5];
  z[0] = v0 * s[0] + v1 * s[1] + v2 * s[2];
  z[1] = v1 * s[0] + v3 * s[1] + v4 * s[2];
  z[2] = v2 * s[0] + v4 * s[1] + v5 * s[2];
}

// Tile header of the tile schedule (back-substitution, linearisation): {L0, nl, o0, n} and
// {S0, ns}.
struct TileHdr {
  int L0, nl, o0, n, S0, ns;
};

__device__ __forceinline__ TileHdr load_tile(const Topology& tp, int tile) {
  const int4 a = tp.tile_desc[2 * tile], b = tp.tile_desc[2 * tile + 1];
  return TileHdr{a.x, a.y, a.z, a.w, b.x, b.y};
}

// ---------------------------------------------------------------------------------------
// Shared memory of a group.  The camera phase of the persistent kernel reuses sg as scratch.
template <typename T> struct GroupSmem;

template <> struct __align__(16) GroupSmem<float> {
  float4 tc[kGroupSlots][3];   // current term of each group slot's camera (9 of 12 used)
  float4 acc[kGroupSlots][3];  // the group slots' sums
  float4 sg[kChunkObs][3];     // a chunk's g rows at their camera-sorted positions
  float tail[kChunkObs / 32][4];  // per warp: the scan value at its last lane
  float head[kChunkObs / 32][4];  // per warp: the scan value at the end of its first segment
  uint32_t clist[2][kChunkObs];   // chunk slots, alternating buffers (filled before the
                                  // barrier that ends the previous chunk's slot sums' reads)
};

// FP64 rows of sg: J_p (18 values) and w = J_l z (2) of the observation at each camera-sorted
// position; the odd stride spreads a warp's rows over the banks.
constexpr int kSgF64 = 21;

template <> struct __align__(16) GroupSmem<double> {
  double2 tc[kGroupSlotsF64][5];  // 9 of 10 used
  double acc[kGroupSlotsF64][9];
  double sg[kChunkObs][kSgF64];   // J_p and w rows at their camera-sorted positions
  double sv[kChunkObs][3];        // each observation's landmark contribution J_l^T J_p t
  double sz[kChunkObs][3];        // z of each landmark of the chunk
};

// Lanes of a chunk's slot sums.  Each of `items` sums (chunk slots are ordered longest first,
// so items are too) runs over `split` lanes, a power of two: the largest s <= 8 with
// items * s <= kChunkObs for every item, and, with the lanes left over, 2 s for the first
// items.  The plan depends on the item count alone, so every sum has a fixed order.
struct SumPlan {
  int s, up;    // base split; items 0 .. up-1 run over 2 s lanes
  int lanes;    // lanes in use
};
__device__ __forceinline__ SumPlan sum_plan(int items) {
  const int s = items * 8 <= kChunkObs ? 8 : items * 4 <= kChunkObs ? 4
              : items * 2 <= kChunkObs ? 2 : 1;
  int up = 0;
  if (s < 16 && items * s < kChunkObs) up = min(items, (kChunkObs - items * s) / s);
  return SumPlan{s, up, items * s + up * s};
}
// Lane idx of the plan: its item, its part (0 .. split-1) and the item's split.
__device__ __forceinline__ void sum_lane(const SumPlan& P, int idx, int& item, int& part,
                                         int& split) {
  const int s2 = 2 * P.s;
  if (idx < P.up * s2) {
    item = idx / s2;
    part = idx - item * s2;
    split = s2;
  } else {
    const int l = idx - P.up * s2;
    item = P.up + l / P.s;
    part = l - (item - P.up) * P.s;
    split = P.s;
  }
}

// ---------------------------------------------------------------------------------------
// FP32-bulk chunk.  Landmark sums: a segmented inclusive scan of v over each warp's lanes
// (shuffles, log2 of the longest segment piece in the warp steps), then, for landmarks that
// cross a warp boundary, the pieces of the warps they span added in warp order (per-warp tail
// and head values in shared memory).  Every observation of a landmark ends with the same sum
// and forms z itself.  Camera sums: g goes to the observation's camera-sorted position; each
// (chunk slot, 4-component quarter) is summed over its rows (split over lanes by sum_plan) and
// added to the group slot's accumulator.  Two block barriers per chunk.
//
// A chunk's inputs reach the threads in one of two ways with the same arithmetic afterwards:
// direct loads from global memory (f32_load_direct), or from a copy of the chunk staged in
// shared memory by bulk asynchronous copies issued one chunk ahead (f32_load_staged).

// Debug builds (checks.cuh): a chunk's indices against their bounds -- an observation code
// (position < n, group slot < gns, the group's slots, landmark < nl), a chunk slot entry (group slot,
// rows [beg, beg + len) within the chunk) and a landmark segment [a, b) -- with out-of-range
// fields replaced by in-range ones.  Release builds return the values unchanged.
__device__ __forceinline__ uint32_t chk_code(const Topology& tp, uint32_t code, int n, int nl,
                                             int gns) {
  if (!kChecks) return code;
  int pos = (int)(code & 0xff), gs = (int)((code >> 8) & 0xff), lm = (int)((code >> 16) & 0xff);
  POBA_CHK(tp.chk, pos, n, kChkChunkPos);
  POBA_CHK(tp.chk, gs, gns, kChkChunkSlot);
  POBA_CHK(tp.chk, lm, nl, kChkChunkLm);
  return (uint32_t)pos | ((uint32_t)gs << 8) | ((uint32_t)lm << 16);
}
__device__ __forceinline__ uint32_t chk_clist(const Topology& tp, uint32_t e, int n, int gns) {
  if (!kChecks) return e;
  int gs = (int)(e & 0xff), beg = (int)((e >> 8) & 0xff), len = (int)(e >> 16);
  POBA_CHK(tp.chk, gs, gns, kChkClistSlot);
  if (len < 1 || beg + len > n) {
    int bad = beg + len;
    POBA_CHK(tp.chk, bad, 0, kChkClistSeg);
    beg = 0;
    len = 0;
  }
  return (uint32_t)gs | ((uint32_t)beg << 8) | ((uint32_t)len << 16);
}
__device__ __forceinline__ void chk_seg(const Topology& tp, int& a, int& b, int n) {
  if (!kChecks) return;
  if (a < 0 || b < a || b > n) {
    int bad = b > n ? b : a;
    POBA_CHK(tp.chk, bad, 0, kChkChunkSeg);
    a = 0;
    b = 0;
  }
}

// One observation thread's inputs.
struct F32Obs {
  float jp[18], jl[6], vi[6];
  uint32_t code;
  int a, b;      // the landmark's segment in the chunk (an inactive lane: [tid, tid + 1))
  uint32_t cl;   // chunk slot tid (threads tid < ns)
};

__device__ __forceinline__ void f32_clear(F32Obs& x) {
#pragma unroll
  for (int k = 0; k < 18; ++k) x.jp[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 6; ++k) x.jl[k] = x.vi[k] = 0.f;
  x.code = 0;
  x.a = threadIdx.x;
  x.b = threadIdx.x + 1;
}

// Sum of rows [beg + part, end) step `split` of column q of sg, in row order; the loads go out
// four at a time ahead of the adds, which stay in row order.
__device__ __forceinline__ float4 sg_rows_sum(const float4 (*sg)[3], int beg, int end, int split,
                                              int q) {
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  int r = beg;
  for (; r + 3 * split < end; r += 4 * split) {
    const float4 v0 = sg[r][q], v1 = sg[r + split][q], v2 = sg[r + 2 * split][q],
                 v3 = sg[r + 3 * split][q];
    s.x += v0.x; s.y += v0.y; s.z += v0.z; s.w += v0.w;
    s.x += v1.x; s.y += v1.y; s.z += v1.z; s.w += v1.w;
    s.x += v2.x; s.y += v2.y; s.z += v2.z; s.w += v2.w;
    s.x += v3.x; s.y += v3.y; s.z += v3.z; s.w += v3.w;
  }
  for (; r < end; r += split) {
    const float4 v = sg[r][q];
    s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
  }
  return s;
}

__device__ __forceinline__ void f32_vinv(F32Obs& x, const float* __restrict__ row) {
  const float2* v2 = reinterpret_cast<const float2*>(row);
  const float2 x0 = v2[0], x1 = v2[1], x2 = v2[2];
  x.vi[0] = x0.x; x.vi[1] = x0.y; x.vi[2] = x1.x; x.vi[3] = x1.y; x.vi[4] = x2.x; x.vi[5] = x2.y;
}

// Chunk c's inputs from global memory (active threads).
__device__ __forceinline__ void f32_load_direct(const Topology& tp, const int4& d0,
                                                const uint8_t* __restrict__ rec,
                                                const ChunkRecLayout& L,
                                                const float* __restrict__ J,
                                                const float* __restrict__ Vinv, F32Obs& x,
                                                int gns = 0) {
  const int tid = threadIdx.x;
  load_J(J, (size_t)tp.n_obs_pad, d0.x + tid, x.jp, x.jl);
  x.code = chk_code(tp, __ldg(reinterpret_cast<const uint32_t*>(rec + L.code) + tid), d0.y, d0.w,
                    gns);
  const int lm = (int)(x.code >> 16) & 0xff;
  const uint16_t* sseg = reinterpret_cast<const uint16_t*>(rec + L.sseg);
  x.a = __ldg(sseg + lm);
  x.b = __ldg(sseg + lm + 1);
  chk_seg(tp, x.a, x.b, d0.y);
  const float2* v2 = reinterpret_cast<const float2*>(Vinv + (size_t)(d0.z + lm) * 6);
  const float2 x0 = __ldg(v2), x1 = __ldg(v2 + 1), x2 = __ldg(v2 + 2);
  x.vi[0] = x0.x; x.vi[1] = x0.y; x.vi[2] = x1.x; x.vi[3] = x1.y; x.vi[4] = x2.x; x.vi[5] = x2.y;
}

// The chunk's computation once each thread holds its inputs (x; RHS mode: (s0, s1, s2) = the
// landmark's b_l).  Threads tid < ns hold chunk slot tid in x.cl, which goes to the shared
// buffer `par` (consecutive chunks of a group alternate 0 and 1).  `ok` is this thread's view of
// whether its inputs are valid (a staged copy that arrived); the barrier after the landmark
// scan reduces it over the block, and if any thread's inputs are invalid every thread returns
// false there, before the hook and before anything is written outside the block's scratch.
// hook() runs right after that barrier (every thread of the block has its inputs in registers
// and has copied the slot list).  Every thread of the block must call it.
template <int MODE, typename Hook>
__device__ __forceinline__ bool chunk_f32_core(const F32Obs& x, bool active, int n, int ns,
                                               int par, float s0, float s1, float s2, bool ok,
                                               GroupSmem<float>& sm, Hook&& hook) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int a = x.a, b = x.b;
  uint32_t* cl = sm.clist[par];
  if (tid < ns) cl[tid] = x.cl;
  const int wb0 = warp * 32;
  const int sb = min(b, wb0 + 32) - wb0;
  float e0 = 0.f, e1 = 0.f, e2 = 0.f;
  if (MODE == kModeSeries) {
    // phase 1: u = J_p t, v = J_l^T u
    if (active) {
      const int gs = (int)(x.code >> 8) & 0xff;
      const float4 ta = sm.tc[gs][0], tb = sm.tc[gs][1], tq = sm.tc[gs][2];
      const float t[9] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w, tq.x};
      float u0 = 0.f, u1 = 0.f;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        u0 += x.jp[j] * t[j];
        u1 += x.jp[9 + j] * t[j];
      }
      s0 = x.jl[0] * u0 + x.jl[3] * u1;
      s1 = x.jl[1] * u0 + x.jl[4] * u1;
      s2 = x.jl[2] * u0 + x.jl[5] * u1;
    }
    // phase 2: segmented scan over the warp's lanes [sa, sb) of each segment
    const int sa = max(a, wb0) - wb0;
    const int span = (int)__reduce_max_sync(kFull, (unsigned)(sb - sa));
    for (int d = 1; d < span; d <<= 1) {
      const float y0 = __shfl_up_sync(kFull, s0, d);
      const float y1 = __shfl_up_sync(kFull, s1, d);
      const float y2 = __shfl_up_sync(kFull, s2, d);
      if (lane - d >= sa) {
        s0 += y0;
        s1 += y1;
        s2 += y2;
      }
    }
    if (lane == 31) {
      sm.tail[warp][0] = s0;
      sm.tail[warp][1] = s1;
      sm.tail[warp][2] = s2;
    }
    if (a < wb0 && lane == sb - 1) {
      sm.head[warp][0] = s0;
      sm.head[warp][1] = s1;
      sm.head[warp][2] = s2;
    }
    e0 = __shfl_sync(kFull, s0, sb - 1);
    e1 = __shfl_sync(kFull, s1, sb - 1);
    e2 = __shfl_sync(kFull, s2, sb - 1);
  }
  // every thread holds its inputs and has finished the previous chunk's slot sums (which read
  // sg and the slot list)
  if (__syncthreads_or(!ok)) return false;
  hook();
  if (MODE == kModeSeries) {
    if (a < wb0 || b > wb0 + 32) {
      // the landmark spans warps wa..wz: tails of wa..wz-1, then the head of wz
      const int wa = min(a >> 5, kChunkObs / 32 - 1), wz = min((b - 1) >> 5, kChunkObs / 32 - 1);
      s0 = s1 = s2 = 0.f;
      for (int w = wa; w < wz; ++w) {
        s0 += sm.tail[w][0];
        s1 += sm.tail[w][1];
        s2 += sm.tail[w][2];
      }
      s0 += sm.head[wz][0];
      s1 += sm.head[wz][1];
      s2 += sm.head[wz][2];
    } else {
      s0 = e0;
      s1 = e1;
      s2 = e2;
    }
  }
  // z = V^-1 s, then g = J_p^T (J_l z) at the camera-sorted position
  if (active) {
    const float z0 = x.vi[0] * s0 + x.vi[1] * s1 + x.vi[2] * s2;
    const float z1 = x.vi[1] * s0 + x.vi[3] * s1 + x.vi[4] * s2;
    const float z2 = x.vi[2] * s0 + x.vi[4] * s1 + x.vi[5] * s2;
    const float w0 = x.jl[0] * z0 + x.jl[1] * z1 + x.jl[2] * z2;
    const float w1 = x.jl[3] * z0 + x.jl[4] * z1 + x.jl[5] * z2;
    float g[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = x.jp[j] * w0 + x.jp[9 + j] * w1;
    float4* row = sm.sg[x.code & 0xff];
    row[0] = make_float4(g[0], g[1], g[2], g[3]);
    row[1] = make_float4(g[4], g[5], g[6], g[7]);
    row[2] = make_float4(g[8], 0.f, 0.f, 0.f);
  }
  __syncthreads();
  // phase 3: chunk slot j (longest first), quarter q: its rows in row order over `split`
  // lanes (sum_plan), combined by a fixed shuffle tree, added to the group slot
  const int items = ns * 3;
  const SumPlan P = sum_plan(items);
  const int bound = (P.lanes + 31) & ~31;
  for (int idx = tid; idx < bound; idx += kChunkObs) {
    int item, part, split;
    sum_lane(P, idx, item, part, split);
    const bool act = idx < P.lanes;
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    int gs = 0, q = 0;
    if (act) {
      const int j = item / 3;
      q = item - 3 * j;
      const uint32_t e = cl[j];
      gs = (int)(e & 0xff);
      const int beg = (int)(e >> 8) & 0xff, end = beg + (int)(e >> 16);
      sum = sg_rows_sum(sm.sg, beg + part, end, split, q);
    }
    for (int off = P.s; off > 0; off >>= 1) {  // levels of the largest split (2 s)
      const float ax = __shfl_down_sync(kFull, sum.x, off);
      const float ay = __shfl_down_sync(kFull, sum.y, off);
      const float az = __shfl_down_sync(kFull, sum.z, off);
      const float aw = __shfl_down_sync(kFull, sum.w, off);
      if (off < split) {
        sum.x += ax;
        sum.y += ay;
        sum.z += az;
        sum.w += aw;
      }
    }
    if (act && part == 0) {
      float4 acc = sm.acc[gs][q];
      acc.x += sum.x;
      acc.y += sum.y;
      acc.z += sum.z;
      acc.w += sum.w;
      sm.acc[gs][q] = acc;
    }
  }
  (void)n;
  return true;
}

// One chunk with direct loads.  Every thread of the block must call it.
template <int MODE>
__device__ __forceinline__ void chunk_f32(const Topology& tp, const SerTopo& sp, int c,
                                          const float* __restrict__ J,
                                          const double* __restrict__ b_l,
                                          const float* __restrict__ Vinv, GroupSmem<float>& sm,
                                          int gns) {
  const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
  const int n = d0.y, ns = d1.x;
  const uint8_t* rec = sp.rec + (size_t)d1.y * 16;
  const ChunkRecLayout L = chunk_rec_layout(n, d0.w, ns);
  const bool active = threadIdx.x < n;
  F32Obs x;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f;
  const uint32_t cl =
      threadIdx.x < ns
          ? chk_clist(tp, __ldg(reinterpret_cast<const uint32_t*>(rec + L.clist) + threadIdx.x), n,
                      gns)
          : 0u;
  if (active) {
    f32_load_direct(tp, d0, rec, L, J, Vinv, x, gns);
    if (MODE == kModeRhs) {
      const double* bl = b_l + (size_t)(d0.z + ((x.code >> 16) & 0xff)) * 3;
      s0 = (float)__ldg(bl);
      s1 = (float)__ldg(bl + 1);
      s2 = (float)__ldg(bl + 2);
    }
  } else {
    f32_clear(x);
  }
  x.cl = cl;
  chunk_f32_core<MODE>(x, active, n, ns, c & 1, s0, s1, s2, true, sm, [] {});
}

// ---------------------------------------------------------------------------------------
// FP64 chunk.  FP64 instructions are the bound here (GB300 runs a warp's FP64 instruction over
// 16 cycles of its FP64 pipe), so the landmark sums use one thread per landmark, which adds
// each contribution once (a scan would add log2 of the track length times), z is formed once
// per landmark, and g = J_p^T w is never formed on its own: each observation leaves J_p and w
// at its camera-sorted position and the lanes of a slot sum accumulate J_p^T w row by row with
// two FMAs per row and component (18 FP64 operations per observation where forming g and then
// adding it took 27).  Three block barriers per chunk.  Every thread must call it.
template <int MODE>
__device__ __forceinline__ void chunk_f64(const Topology& tp, const SerTopo& sp, int c,
                                          const double* __restrict__ J,
                                          const double* __restrict__ b_l,
                                          const double* __restrict__ Vinv, GroupSmem<double>& sm,
                                          int gns) {
  const int tid = threadIdx.x;
  const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
  const int o0 = d0.x, n = d0.y, L0 = d0.z, nl = d0.w, ns = d1.x;
  const uint8_t* rec = sp.rec + (size_t)d1.y * 16;
  const ChunkRecLayout L = chunk_rec_layout(n, nl, ns);
  const bool active = tid < n;
  double (*sv)[3] = sm.sv;
  double jp[18], jl[6];
  uint32_t code = 0;
  const uint64_t pol = l2_stream_policy();
  if (active) {
    load_J_stream(J, (size_t)tp.n_obs_pad, o0 + tid, jp, jl, pol);
    code = chk_code(tp, ldg_stream(reinterpret_cast<const uint32_t*>(rec + L.code) + tid, pol), n,
                    nl, gns);
  }
  double vi[6], sl[3] = {0.0, 0.0, 0.0};
  int a = 0, b = 0;
  if (tid < nl) {
    const uint16_t* sseg = reinterpret_cast<const uint16_t*>(rec + L.sseg);
    a = __ldg(sseg + tid);
    b = __ldg(sseg + tid + 1);
    chk_seg(tp, a, b, n);
    const double2* v2 = reinterpret_cast<const double2*>(Vinv + (size_t)(L0 + tid) * 6);
    const double2 x0 = ldg_stream(v2, pol), x1 = ldg_stream(v2 + 1, pol), x2 = ldg_stream(v2 + 2, pol);
    vi[0] = x0.x; vi[1] = x0.y; vi[2] = x1.x; vi[3] = x1.y; vi[4] = x2.x; vi[5] = x2.y;
    if (MODE == kModeRhs) {
      const double* bl = b_l + (size_t)(L0 + tid) * 3;
      sl[0] = __ldg(bl);
      sl[1] = __ldg(bl + 1);
      sl[2] = __ldg(bl + 2);
    }
  }
  if (MODE == kModeSeries) {
    if (active) {
      const int gs = (int)(code >> 8) & 0xff;
      const double* tc = reinterpret_cast<const double*>(sm.tc[gs]);
      double u0 = 0.0, u1 = 0.0;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        u0 += jp[j] * tc[j];
        u1 += jp[9 + j] * tc[j];
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) sv[tid][k] = jl[k] * u0 + jl[3 + k] * u1;
    }
    __syncthreads();
    if (tid < nl) {
      for (int q = a; q < b; ++q) {
        sl[0] += sv[q][0];
        sl[1] += sv[q][1];
        sl[2] += sv[q][2];
      }
    }
  }
  if (tid < nl) {
    double z[3];
    apply_vinv(vi, sl, z);
    sm.sz[tid][0] = z[0];
    sm.sz[tid][1] = z[1];
    sm.sz[tid][2] = z[2];
  }
  __syncthreads();
  if (active) {
    const int lm = (int)(code >> 16) & 0xff;
    const double z0 = sm.sz[lm][0], z1 = sm.sz[lm][1], z2 = sm.sz[lm][2];
    const double w0 = jl[0] * z0 + jl[1] * z1 + jl[2] * z2;
    const double w1 = jl[3] * z0 + jl[4] * z1 + jl[5] * z2;
    double* row = sm.sg[code & 0xff];
#pragma unroll
    for (int k = 0; k < 18; ++k) row[k] = jp[k];
    row[18] = w0;
    row[19] = w1;
  }
  __syncthreads();
  // chunk slot j, component k: sum over rows [beg_j, beg_{j+1}) (over `split` lanes) of
  // J_p[k] w0 + J_p[9 + k] w1, then the group slot
  const uint32_t* clist = reinterpret_cast<const uint32_t*>(rec + L.clist);
  const int items = ns * 9;
  const SumPlan P = sum_plan(items);
  const int bound = (P.lanes + 31) & ~31;
  for (int idx = tid; idx < bound; idx += kChunkObs) {
    int item, part, split;
    sum_lane(P, idx, item, part, split);
    const bool act = idx < P.lanes;
    double s = 0.0;
    int gs = 0, k = 0;
    if (act) {
      const int j = item / 9;
      k = item - 9 * j;
      const uint32_t e = chk_clist(tp, __ldg(clist + j), n, gns);
      gs = (int)(e & 0xff);
      const int beg = (int)(e >> 8) & 0xff, end = beg + (int)(e >> 16);
      for (int r = beg + part; r < end; r += split) {
        const double* q = sm.sg[r];
        s = __fma_rn(q[k], q[18], s);
        s = __fma_rn(q[9 + k], q[19], s);
      }
    }
    for (int off = P.s; off > 0; off >>= 1) {  // levels of the largest split (2 s)
      const double a = __shfl_down_sync(kFull, s, off);
      if (off < split) s += a;
    }
    if (act && part == 0) sm.acc[gs][k] += s;
  }
}

// The group of a long track (more than kChunkObs observations; its pieces are the group's
// chunks, one internal landmark each, every piece holding the track's V^-1 and b_l).  Series
// mode, pass A: per piece, thread o forms v_o = J_l,o^T J_p,o t_c(o) and the block sums the
// piece's v in a fixed order (block_sum_tile, in double); the piece sums are added in piece
// order (in double); z = V^-1 of that sum.  RHS mode: z = V^-1 b_l.  Pass B, per piece: g_o =
// J_p,o^T (J_l,o z) at its camera-sorted position, then thread (slot, k) sums its slot's rows
// in order and writes the piece's own partial row for that slot (a long group keeps no
// accumulator across its chunks).  J is read twice in series mode.  Every thread must call it.
template <typename T, int MODE>
__device__ __noinline__ void long_group_body(const Topology& tp, const SerTopo& sp, int g,
                                             const T* __restrict__ J,
                                             const T* __restrict__ t_cam,
                                             const double* __restrict__ b_l,
                                             const T* __restrict__ Vinv, T* __restrict__ partial,
                                             GroupSmem<T>& sm) {
  const int tid = threadIdx.x;
  const int4 gd = __ldg(sp.group + 2 * g);
  const int c0 = gd.x, nc = gd.y, s0 = gd.z;
  double* sbuf = reinterpret_cast<double*>(&sm.acc[0][0]);  // kChunkObs doubles
  T (*rows)[9] = reinterpret_cast<T (*)[9]>(&sm.sg[0][0]);  // kChunkObs rows
  __shared__ double zs[3];
  const size_t pad = (size_t)tp.n_obs_pad;
  const int L = __ldg(sp.chunk + 2 * c0).z;  // the first piece (all pieces hold the same V^-1)
  double S0 = 0.0, S1 = 0.0, S2 = 0.0;
  if (MODE == kModeSeries) {
    for (int c = c0; c < c0 + nc; ++c) {
      const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
      const int o0 = d0.x, n = d0.y, sbase = d1.w;
      const uint8_t* rec = sp.rec + (size_t)d1.y * 16;
      double v0 = 0.0, v1 = 0.0, v2 = 0.0;
      if (tid < n) {
        T jp[18], jl[6];
        load_J(J, pad, o0 + tid, jp, jl);
        const uint32_t code = __ldg(reinterpret_cast<const uint32_t*>(rec) + tid);
        const int cam = __ldg(sp.gslot_cam + s0 + sbase + (int)((code >> 8) & 0xff));
        const T* tc = t_cam + (size_t)cam * kTStride;
        T u0 = (T)0, u1 = (T)0;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
          const T tj = __ldcg(tc + j);
          u0 += jp[j] * tj;
          u1 += jp[9 + j] * tj;
        }
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
  } else if (tid == 0) {
    S0 = b_l[(size_t)L * 3 + 0];
    S1 = b_l[(size_t)L * 3 + 1];
    S2 = b_l[(size_t)L * 3 + 2];
  }
  if (tid == 0) {
    const T* vi = Vinv + (size_t)L * 6;
    const double w0 = (double)vi[0], w1 = (double)vi[1], w2 = (double)vi[2];
    const double w3 = (double)vi[3], w4 = (double)vi[4], w5 = (double)vi[5];
    zs[0] = w0 * S0 + w1 * S1 + w2 * S2;
    zs[1] = w1 * S0 + w3 * S1 + w4 * S2;
    zs[2] = w2 * S0 + w4 * S1 + w5 * S2;
  }
  __syncthreads();
  const T z0 = (T)zs[0], z1 = (T)zs[1], z2 = (T)zs[2];
  for (int c = c0; c < c0 + nc; ++c) {
    const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
    const int o0 = d0.x, n = d0.y, ns = d1.x, sbase = d1.w;
    const uint8_t* rec = sp.rec + (size_t)d1.y * 16;
    const ChunkRecLayout RL = chunk_rec_layout(n, 1, ns);
    if (tid < n) {
      T jp[18], jl[6];
      load_J(J, pad, o0 + tid, jp, jl);
      const uint32_t code = __ldg(reinterpret_cast<const uint32_t*>(rec + RL.code) + tid);
      const T w0 = jl[0] * z0 + jl[1] * z1 + jl[2] * z2;
      const T w1 = jl[3] * z0 + jl[4] * z1 + jl[5] * z2;
      T* row = rows[code & 0xff];
#pragma unroll
      for (int k = 0; k < 9; ++k) row[k] = jp[k] * w0 + jp[9 + k] * w1;
    }
    __syncthreads();
    const uint32_t* clist = reinterpret_cast<const uint32_t*>(rec + RL.clist);
    for (int i = tid; i < ns * 9; i += blockDim.x) {
      const int j = i / 9, k = i - 9 * j;
      const uint32_t e = __ldg(clist + j);
      const int gs = (int)(e & 0xff), beg = (int)(e >> 8) & 0xff, len = (int)(e >> 16);
      T acc = (T)0;
      for (int r = beg; r < beg + len; ++r) acc += rows[r][k];
      partial[(size_t)__ldg(sp.gslot_row + s0 + sbase + gs) * 9 + k] = acc;
    }
    __syncthreads();
  }
}

// Bytes [p, p + bytes) toward L2 (one bulk prefetch; stream: with the streaming policy).  The
// range is widened to 16-byte bounds, which must stay inside the allocation (every arena item
// starts on a 256-byte boundary, so a range within one item qualifies).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes, bool stream) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~(uintptr_t)15;
  if (e <= a) return;
  if (stream)
    asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(a),
                 "r"((unsigned)(e - a)), "l"(l2_stream_policy())
                 : "memory");
  else
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((unsigned)(e - a))
                 : "memory");
}

// Chunks of a group prefetched to L2 ahead of the one the block runs (when the schedule asks for
// it: sp.prefetch, set when the Jacobians take more than half of L2, so that a term streams
// much of them from HBM).
constexpr int kChunkAhead = 1;

// Chunk c's inputs toward L2 ahead of their use: the Jacobian plane groups of its observations
// (24 / V contiguous ranges of n 16-byte groups), its record and the V^-1 rows of its landmarks,
// one bulk prefetch per range, issued by the first lanes of the calling warp (FP64: with the
// streaming policy of the FP64 chunk's loads).  A prefetch changes no data, so the chunk's sums
// are the same with or without it.
template <typename T>
__device__ __forceinline__ void prefetch_chunk_l2(const Topology& tp, const SerTopo& sp, int c,
                                                  const T* __restrict__ J,
                                                  const T* __restrict__ Vinv, int lane) {
  constexpr int V = jgroup<T>(), NG = 24 / V;
  if (lane >= NG + 2) return;
  const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
  const char* p;
  size_t bytes;
  if (lane < NG) {
    p = reinterpret_cast<const char*>(jgroups(J) + (size_t)lane * tp.n_obs_pad + d0.x);
    bytes = (size_t)d0.y * 16;
  } else if (lane == NG) {
    p = reinterpret_cast<const char*>(sp.rec + (size_t)d1.y * 16);
    bytes = (size_t)chunk_rec_layout(d0.y, d0.w, d1.x).bytes;
  } else {
    p = reinterpret_cast<const char*>(Vinv + (size_t)d0.z * 6);
    bytes = (size_t)d0.w * 6 * sizeof(T);
  }
  prefetch_l2(p, bytes, sizeof(T) == 8);
}

// One group (blockDim.x == kChunkObs; every thread must call it, and every thread must have
// finished with the shared memory of the previous group, e.g. by a block barrier): stages the
// current term of the group's slots and zeroes their accumulators, runs the chunks in order and
// writes one partial row per group slot (row gslot_row[s], 9 values in the bulk precision).
template <typename T, int MODE>
__device__ __forceinline__ void group_body(const Topology& tp, const SerTopo& sp, int g,
                                           const T* __restrict__ J,
                                           const T* __restrict__ t_cam,
                                           const double* __restrict__ b_l,
                                           const T* __restrict__ Vinv, T* __restrict__ partial,
                                           GroupSmem<T>& sm) {
  const int tid = threadIdx.x;
  if (__ldg(sp.group + 2 * g + 1).z) {
    long_group_body<T, MODE>(tp, sp, g, J, t_cam, b_l, Vinv, partial, sm);
    return;
  }
  const int4 gd = __ldg(sp.group + 2 * g);
  const int c0 = gd.x, nc = gd.y, s0 = gd.z, ns = gd.w;
  // the last warp prefetches the first chunks now (their loads overlap the staging of t) and
  // chunk c + kChunkAhead while the block runs chunk c
  const int pw_lane = sp.prefetch ? tid - (kChunkObs - 32) : -1;
  if (pw_lane >= 0)
    for (int c = c0; c < c0 + min(nc, kChunkAhead); ++c)
      prefetch_chunk_l2<T>(tp, sp, c, J, Vinv, pw_lane);
  constexpr int R = sizeof(T) == 4 ? 3 : 5;  // 16-byte pieces of a term row in shared memory
  for (int i = tid; i < ns * R; i += kChunkObs) {
    const int s = i / R, q = i - R * s;
    if constexpr (sizeof(T) == 4) {
      sm.acc[s][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (MODE == kModeSeries) {
        int cam = __ldg(sp.gslot_cam + s0 + s);
        POBA_CHK(tp.chk, cam, tp.n_cams, kChkSerCam);
        sm.tc[s][q] = __ldcg(reinterpret_cast<const float4*>(t_cam + (size_t)cam * kTStride) + q);
      }
    } else {
      if (q < 4) {
        sm.acc[s][2 * q] = 0.0;
        sm.acc[s][2 * q + 1] = 0.0;
      } else {
        sm.acc[s][8] = 0.0;
      }
      if (MODE == kModeSeries) {
        int cam = __ldg(sp.gslot_cam + s0 + s);
        POBA_CHK(tp.chk, cam, tp.n_cams, kChkSerCam);
        const double* src = t_cam + (size_t)cam * kTStride;
        sm.tc[s][q] = q < 4 ? __ldcg(reinterpret_cast<const double2*>(src) + q)
                            : make_double2(__ldcg(src + 8), 0.0);
      }
    }
  }
  __syncthreads();
  if constexpr (sizeof(T) == 4) {
    for (int c = c0; c < c0 + nc; ++c) {
      if (pw_lane >= 0 && c + kChunkAhead < c0 + nc)
        prefetch_chunk_l2<T>(tp, sp, c + kChunkAhead, J, Vinv, pw_lane);
      chunk_f32<MODE>(tp, sp, c, J, b_l, Vinv, sm, ns);
    }
  } else {
    for (int c = c0; c < c0 + nc; ++c) {
      if (pw_lane >= 0 && c + kChunkAhead < c0 + nc)
        prefetch_chunk_l2<T>(tp, sp, c + kChunkAhead, J, Vinv, pw_lane);
      chunk_f64<MODE>(tp, sp, c, J, b_l, Vinv, sm, ns);
    }
  }
  __syncthreads();
  for (int i = tid; i < ns * 9; i += kChunkObs) {
    const int s = i / 9, k = i - 9 * s;
    int row = __ldg(sp.gslot_row + s0 + s);
    POBA_CHK(tp.chk, row, sp.n_gslots, kChkSerRow);
    T v;
    if constexpr (sizeof(T) == 4)
      v = reinterpret_cast<const float*>(sm.acc[s])[k];
    else
      v = sm.acc[s][k];
    partial[(size_t)row * 9 + k] = v;
  }
}

// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}

// Sum of one chunk of a camera's partial rows, component k: rows [q0, q1) in row order (loads
// are issued 16 floats or 8 doubles at a time).  A chunk is a segment: FP32-bulk rows are added
// in float inside it and the chunks in double (camera_body), FP64 rows in double throughout.
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

// One entry of a camera's norm pair: the sum of its 9 squared components in component order
// (every camera update path uses this order).  The camera updates run it on a thread per pair
// entry, packed into the first threads of the block: each FP64 warp instruction costs 16 pipe
// cycles on GB300, so the fewer warps issue these adds the better.
__device__ __forceinline__ double norm_row_sum(const double* sq) {
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < 9; ++j) a += sq[j];
  return a;
}

// Camera body for cameras [cam0, cam0 + per_block): thread (c, k) sums component k of the
// camera's contiguous partial rows [cam_ptr[c], cam_ptr[c + 1]) (chunk by chunk, cam_chunk_rows
// rows per chunk, the chunks in order), applies row k of U^-1, updates x and writes the new term
// t_cam[c]; then the camera's squared term and x components are added (in component order,
// norm_row_sum) into its pair cam_norm[c] = (||t_c||^2, ||x_c||^2).  Cameras of
// problems whose series has stopped are left as they are.  FP64 work is one add per row and
// component: every FP64 warp instruction costs 16 pipe cycles on GB300, so no shuffle trees are
// used for the row sums.  ys and y2 are shared [per_block][9] arrays.  Every thread of the block
// must call it.
template <typename PT, int MODE>
__device__ __forceinline__ void camera_body(const Topology& tp, const int32_t* __restrict__ cam_ptr,
                                            int cam0, int per_block,
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
    int r0 = cam_ptr[c], r1 = cam_ptr[c + 1];
    if (kChecks && (r0 < 0 || r1 < r0 || r1 > cam_ptr[tp.n_cams])) {
      int bad = r1;
      POBA_CHK(tp.chk, bad, 0, kChkCamRows);
      r0 = r1 = 0;
    }
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
  // the norm pairs: the block's first 2 per_block threads, one pair entry each (the done flags
  // cannot change before every block of the launch has passed here)
  if (tid < 2 * per_block) {
    const int cn = tid >> 1, e = tid & 1, cc = cam0 + cn;
    if (cc < tp.n_cams && !ld_volatile(&st[tp.cam_prob[cc]].done))
      cam_norm[2 * cc + e] = norm_row_sum(e ? y2[cn] : ys[cn]);
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

// Sum of the camera norm pairs (||t_c||^2, ||x_c||^2) of cameras [c0, c1), the two sums of the
// stop rule.  The order depends only on the camera count, so every execution form gets the same
// bits: a problem with fewer than kBlockNormCams cameras is summed by one warp (lane j adds
// cameras c0 + j, c0 + j + 32, ... in order, then a fixed shuffle tree); a larger one over
// kNormLanes virtual lanes (lane v adds cameras c0 + v, c0 + v + kNormLanes, ... in order; the
// block's threads run the lanes whatever the block size), whose sums warp 0 combines: lane j
// adds virtual lanes j, j + 32, ..., j + kNormLanes - 32 in order, then the same shuffle tree.
// Loads go out eight at a time.
constexpr int kBlockNormCams = 2048;
constexpr int kNormLanes = 256;

__device__ __forceinline__ void strided_norm_sum(const double2* __restrict__ cn, int c, int c1,
                                                 int stride, double& a, double& b) {
  for (int cb = c; cb < c1; cb += stride * 8) {
    double2 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      v[j] = cb + stride * j < c1 ? __ldcg(cn + cb + stride * j) : make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a += v[j].x;
      b += v[j].y;
    }
  }
}

__device__ __forceinline__ void warp_tree(double& a, double& b) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
}

// One warp (all 32 lanes), a problem below kBlockNormCams cameras; the sums land in lane 0.
__device__ __forceinline__ void warp_norm_sums(const double* __restrict__ cam_norm, int c0, int c1,
                                               double& a, double& b) {
  const int lane = threadIdx.x & 31;
  a = 0.0;
  b = 0.0;
  strided_norm_sum(reinterpret_cast<const double2*>(cam_norm), c0 + lane, c1, 32, a, b);
  warp_tree(a, b);
}

// Every thread of the block (at least one full warp), a problem of at least kBlockNormCams
// cameras; red: 2 kNormLanes doubles of shared scratch.  The sums land in thread 0.
__device__ __forceinline__ void block_norm_sums(const double* __restrict__ cam_norm, int c0, int c1,
                                                double* red, double& a, double& b) {
  const double2* cn = reinterpret_cast<const double2*>(cam_norm);
  for (int v = threadIdx.x; v < kNormLanes; v += blockDim.x) {
    double va = 0.0, vb = 0.0;
    strided_norm_sum(cn, c0 + v, c1, kNormLanes, va, vb);
    red[2 * v] = va;
    red[2 * v + 1] = vb;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  if (threadIdx.x < 32) {
#pragma unroll
    for (int j = 0; j < kNormLanes / 32; ++j) {
      a += red[2 * (threadIdx.x + 32 * j)];
      b += red[2 * (threadIdx.x + 32 * j) + 1];
    }
    warp_tree(a, b);
  }
  __syncthreads();
}

// Every problem still running: sum its cameras' norm pairs and apply its stop rule for term
// `iter`; raise all_done when no problem is left and record the running count.  Problems below
// kBlockNormCams cameras take one warp each (several at once), larger ones the whole block in
// turn.  Every thread of one block (at least one full warp) must call it; red as for
// block_norm_sums.
__device__ __forceinline__ void problems_stop_rule(const Topology& tp,
                                                   const double* __restrict__ cam_norm,
                                                   SeriesState* st, SeriesGlobal* sgl, int iter,
                                                   double eps, int* s_running, double* red) {
  // only full warps take problems (the shuffles use every lane of a warp)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) *s_running = 0;
  __syncthreads();
  for (int p = warp; warp < nw && p < tp.n_probs; p += nw) {
    const int c0 = tp.cam_off[p], c1 = tp.cam_off[p + 1];
    if (c1 - c0 >= kBlockNormCams || ld_volatile(&st[p].done)) continue;  // warp-uniform
    double a, b;
    warp_norm_sums(cam_norm, c0, c1, a, b);
    if (lane == 0) {
      series_stop_rule(&st[p], iter, a, b, eps);
      if (!st[p].done) atomicAdd(s_running, 1);
    }
  }
  for (int p = 0; p < tp.n_probs; ++p) {
    const int c0 = tp.cam_off[p], c1 = tp.cam_off[p + 1];
    if (c1 - c0 < kBlockNormCams) continue;  // block-uniform
    __syncthreads();
    if (ld_volatile(&st[p].done)) continue;  // the same value in every thread (after the barrier)
    double a, b;
    block_norm_sums(cam_norm, c0, c1, red, a, b);
    if (threadIdx.x == 0) {
      series_stop_rule(&st[p], iter, a, b, eps);
      if (!st[p].done) atomicAdd(s_running, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sgl->n_running = *s_running;
    if (*s_running == 0) sgl->all_done = 1;
  }
  __syncthreads();
}

}  // namespace poba
