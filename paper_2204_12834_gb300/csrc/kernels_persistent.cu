// Persistent power-series kernel of libpoba (sm_103a): after the reduced right-hand side and
// x(0) (two per-term launches), one cooperative launch runs every series term and the stop
// rule of Sec. 4.3 (eqs. `S_approx`, `x_approx`, `qcriterion`).
//
// Each term is two phases separated by grid barriers:
//   phase A  every block pulls tiles from a shared counter and runs the tile body (W^T t,
//            V^-1, W z) -- dynamic scheduling, so no wave tail;
//   phase B  camera groups (blockDim / 9 cameras each, static round-robin) run the camera body
//            (U^-1, x accumulation, new term rows) and store per-group squared norms;
//   barrier  the last block to arrive opens it at once, then sums the group norms in group
//            order and applies the stop rule; the other blocks see the decision before their
//            next tile fetch and, at the latest, at the next barrier (a stop skips the camera
//            phase, so x stays at the term where the rule fired).
// Results are bitwise equal to the per-term launches: every tile and camera computes the same
// sums in the same order whichever block runs it.
//
// Every barrier wait is bounded: after `timeout` clock cycles a block sets the error flag and
// all blocks leave at their next barrier (the host reports BA_ERR_TIMEOUT).
#include <cmath>

#include "poba_internal.cuh"
#include "series_body.cuh"
#include "tile_common.cuh"

namespace poba {

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// Arrive at the barrier.  Returns (in every thread) whether this block arrived last; the
// generation seen before arriving is stored in *gen.
__device__ __forceinline__ int barrier_arrive(GridSync* gs, unsigned G, unsigned* gen, int* s_last,
                                              unsigned* s_gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_volatile(&gs->gen);
    __threadfence();
    const unsigned ticket = atomicAdd(&gs->count, 1u);
    *s_last = ticket == G - 1;
    *s_gen = g;
  }
  __syncthreads();
  *gen = *s_gen;
  return *s_last;
}

// Last block: open the barrier (after its own work).  Thread 0 only.
__device__ __forceinline__ void barrier_release(GridSync* gs) {
  gs->count = 0u;
  __threadfence();
  atomicAdd(&gs->gen, 1u);
}

// Wait until the generation moves past `gen`; false on timeout or when another block failed.
// Polls with an exponential back-off (32 ns .. 512 ns) to keep the hot word quiet.
__device__ __forceinline__ bool barrier_wait(GridSync* gs, unsigned gen, long long timeout,
                                             int* s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    unsigned sleep_ns = 32;
    for (unsigned it = 0; ld_volatile(&gs->gen) == gen; ++it) {
      if (clock64() - t0 > timeout) {
        atomicExch(&gs->error, 1);
        ok = 0;
        break;
      }
      if ((it & 15u) == 15u && ld_volatile(&gs->error)) {
        ok = 0;
        break;
      }
      __nanosleep(sleep_ns);
      if (sleep_ns < 512) sleep_ns <<= 1;
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(kTileObs, sizeof(T) == 8 ? 3 : 3) series_persistent_kernel(
    Topology tp, const T* __restrict__ J, const T* __restrict__ Vinv,
    const double* __restrict__ b_l, const double* __restrict__ b_p,
    const double* __restrict__ Uinv, double* __restrict__ x, T* __restrict__ t_cm,
    T* __restrict__ partial, double* __restrict__ group_norms, SeriesState* __restrict__ st,
    GridSync* __restrict__ gs, int m_max, double eps, long long timeout,
    long long* __restrict__ trace) {
  __shared__ TileSmem<T> sm;
  __shared__ double sred[kTileObs / 32];
  __shared__ int s_tile, s_last, s_ok, s_done;
  __shared__ unsigned s_gen;
  const int tid = threadIdx.x;
  const unsigned G = gridDim.x;
  // camera groups: spread over every block (cameras per group = ceil(n_cams / blocks), at most
  // blockDim / 9), so the FP64 camera work of a term runs on all SMs at once
  const int cap = kTileObs / 9;
  int per_group = (tp.n_cams + (int)G - 1) / (int)G;
  per_group = per_group < 1 ? 1 : (per_group > cap ? cap : per_group);
  const int n_groups = (tp.n_cams + per_group - 1) / per_group;
  double (*ys)[9] = reinterpret_cast<double (*)[9]>(&sm.sg[0][0]);  // phase B reuses sg

  if (tid == 0) s_done = ld_volatile(&st->done);  // x(0) = 0 stops before the first term
  __syncthreads();
  if (s_done) return;
  // the block's first camera group is fixed for the whole launch: keep its slot-row range and
  // its components of x in registers (x is written back once at the end)
  const int c_cl = tid / 9, ck = tid - c_cl * 9;
  const int c0 = blockIdx.x * per_group + c_cl;
  const bool c_ok = (int)blockIdx.x < n_groups && c_cl < per_group && c0 < tp.n_cams;
  int c_r0 = 0, c_r1 = 0;
  double x_reg = 0.0;
  if (c_ok) {
    c_r0 = tp.cam_slot_ptr[c0];
    c_r1 = tp.cam_slot_ptr[c0 + 1];
    x_reg = x[(size_t)c0 * 9 + ck];
  }
  const bool tracer = blockIdx.x == 0 && tid == 0 && trace != nullptr;
  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    // ---- phase A: tiles (the next tile index is fetched while the current one is processed;
    // a stop decided for the previous term makes the remaining tiles of this one moot)
    int next = 0;
    if (tid == 0) next = ld_volatile(&st->done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
    for (;;) {
      if (tid == 0) {
        s_tile = next;
        if (next < tp.n_tiles)
          next = ld_volatile(&st->done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
      }
      __syncthreads();
      const int tile = s_tile;
      __syncthreads();
      if (tile >= tp.n_tiles) break;
      if constexpr (sizeof(T) == 4)
        tile_matvec_body_f32<kModeSeries>(tp, tile, J, t_cm, b_l, Vinv, partial, sm);
      else
        tile_matvec_body<T, kModeSeries>(tp, tile, J, t_cm, b_l, Vinv, partial, sm);
    }
    unsigned gen;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 1] = global_ns();
    if (barrier_arrive(gs, G, &gen, &s_last, &s_gen)) {
      if (tid == 0) {
        gs->tile_next = 0u;
        barrier_release(gs);
      }
    } else if (!barrier_wait(gs, gen, timeout, &s_ok)) {
      return;
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 2] = global_ns();
    if (tid == 0) s_done = ld_volatile(&st->done);
    __syncthreads();
    if (s_done) break;  // the rule fired at term i - 1: x stays x(i - 1)
    // ---- phase B: cameras (the block's first group uses the cached rows and x)
    for (int g = blockIdx.x; g < n_groups; g += G) {
      double v, xv;
      if (g == (int)blockIdx.x) {
        double ui[9];
        if (c_ok) {
#pragma unroll
          for (int j = 0; j < 9; ++j) ui[j] = Uinv[(size_t)c0 * 81 + ck * 9 + j];
        }
        double y = 0.0;
        for (int rb = c_r0; rb < c_r1; rb += 8) {
          T buf[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) buf[j] = (rb + j < c_r1) ? __ldcg(partial + (size_t)(rb + j) * 9 + ck) : (T)0;
#pragma unroll
          for (int j = 0; j < 8; ++j) y += (double)buf[j];
        }
        if (c_cl < per_group) ys[c_cl][ck] = y;
        __syncthreads();
        v = 0.0;
        xv = 0.0;
        if (c_ok) {
#pragma unroll
          for (int j = 0; j < 9; ++j) v += ui[j] * ys[c_cl][j];
          x_reg += v;
          xv = x_reg;
          const T tv = (T)v;
          for (int q = c_r0; q < c_r1; ++q) t_cm[(size_t)q * 9 + ck] = tv;
        }
      } else {
        camera_body<T, kModeSeries>(tp, g * per_group, per_group, partial, b_p, Uinv, x, t_cm,
                                    ys, v, xv);
      }
      const double bt = block_sum_fixed(v * v, sred);
      __syncthreads();
      const double bx = block_sum_fixed(xv * xv, sred);
      if (tid == 0) {
        group_norms[2 * g + 0] = bt;
        group_norms[2 * g + 1] = bx;
      }
      __syncthreads();
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (barrier_arrive(gs, G, &gen, &s_last, &s_gen)) {
      // last block: open the barrier, then the norms in group order and the stop rule for
      // term i (visible to every block before the next barrier)
      if (tid == 0) barrier_release(gs);
      __threadfence();
      double at = 0.0, ax = 0.0;
      for (int g = tid; g < n_groups; g += blockDim.x) {
        at += __ldcg(group_norms + 2 * g + 0);
        ax += __ldcg(group_norms + 2 * g + 1);
      }
      const double T2 = block_sum_fixed(at, sred);
      __syncthreads();
      const double X2 = block_sum_fixed(ax, sred);
      if (tid == 0) {
        series_stop_rule(st, i, T2, X2, eps);
        __threadfence();
      }
      __syncthreads();
    } else if (!barrier_wait(gs, gen, timeout, &s_ok)) {
      return;
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  if (c_ok) x[(size_t)c0 * 9 + ck] = x_reg;
}

int persistent_blocks_per_sm(bool f32) {
  int nb = 0;
  if (f32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_kernel<float>, kTileObs, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_kernel<double>, kTileObs, 0);
  return nb;
}

template <typename T>
cudaError_t launch_series_persistent(const Topology& tp, int grid, const T* J, const T* Vinv,
                                     const double* b_l, const double* b_p, const double* Uinv,
                                     double* x, T* t_cm, T* partial, double* group_norms,
                                     SeriesState* st, GridSync* gs, int m_max, double eps,
                                     long long timeout, long long* trace, cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&J, (void*)&Vinv, (void*)&b_l, (void*)&b_p, (void*)&Uinv,
                  (void*)&x, (void*)&t_cm, (void*)&partial, (void*)&group_norms, (void*)&st,
                  (void*)&gs, (void*)&m_max, (void*)&eps, (void*)&timeout, (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_persistent_kernel<T>, dim3(grid),
                                     dim3(kTileObs), args, 0, s);
}

template cudaError_t launch_series_persistent<double>(const Topology&, int, const double*, const double*, const double*, const double*, const double*, double*, double*, double*, double*, SeriesState*, GridSync*, int, double, long long, long long*, cudaStream_t);
template cudaError_t launch_series_persistent<float>(const Topology&, int, const float*, const float*, const double*, const double*, const double*, double*, float*, float*, double*, SeriesState*, GridSync*, int, double, long long, long long*, cudaStream_t);

}  // namespace poba
