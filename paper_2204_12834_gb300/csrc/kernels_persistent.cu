// Persistent power-series kernel of libpoba (sm_103a): after the reduced right-hand side and
// x(0) (two per-term launches), one cooperative launch runs every series term and the stop
// rule of Sec. 4.3 (eqs. `S_approx`, `x_approx`, `qcriterion`).
//
// Each term is two phases separated by grid barriers:
//   phase A  every block pulls tiles from a shared counter and runs the tile body (W^T t,
//            V^-1, W z) -- dynamic scheduling, so no wave tail;
//   phase B  camera groups (spread over all blocks, static) run the camera body (U^-1, x
//            accumulation, new term rows) and store a squared-norm pair per camera;
//   barrier  the last block to arrive opens it at once, then sums each running problem's
//            camera norm pairs in camera order and applies its stop rule; the other blocks see
//            the decisions before their next tile fetch and, at the latest, at the next
//            barrier (a stopped problem's tiles and cameras are skipped, so its x stays at the
//            term where its rule fired).
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
__global__ void __launch_bounds__(kTileObs, 3) series_persistent_kernel(
    Topology tp, const T* __restrict__ J, const T* __restrict__ Vinv,
    const double* __restrict__ Uinv, double* __restrict__ x, T* __restrict__ t_cm,
    T* __restrict__ partial, double* __restrict__ cam_norm, SeriesState* __restrict__ st,
    SeriesGlobal* __restrict__ sgl, GridSync* __restrict__ gs, int m_max, double eps,
    long long timeout, long long* __restrict__ trace) {
  __shared__ TileSmem<T> sm;
  __shared__ int s_tile, s_last, s_ok, s_done, s_running;
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
  double (*y2)[9] = ys + cap;

  if (tid == 0) s_done = ld_volatile(&sgl->all_done);  // every x(0) = 0: nothing to do
  __syncthreads();
  if (s_done) return;
  // the block's first camera group is fixed for the whole launch: keep its slot-row range and
  // its components of x in registers (x is written back once at the end)
  const int c_cl = tid / 9, ck = tid - c_cl * 9;
  const int c0 = blockIdx.x * per_group + c_cl;
  const bool c_mine = (int)blockIdx.x < n_groups && c_cl < per_group && c0 < tp.n_cams;
  int c_r0 = 0, c_r1 = 0, c_prob = 0;
  double x_reg = 0.0;
  if (c_mine) {
    c_r0 = tp.cam_slot_ptr[c0];
    c_r1 = tp.cam_slot_ptr[c0 + 1];
    c_prob = tp.cam_prob[c0];
    x_reg = x[(size_t)c0 * 9 + ck];
  }
  const bool tracer = blockIdx.x == 0 && tid == 0 && trace != nullptr;
  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    // ---- phase A: tiles (the next tile index is fetched while the current one is processed;
    // once every problem has stopped the remaining tiles are moot; tiles of a problem that
    // stopped are skipped)
    int next = 0;
    if (tid == 0)
      next = ld_volatile(&sgl->all_done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
    for (;;) {
      if (tid == 0) {
        int cur = next;
        while (cur < tp.n_tiles && ld_volatile(&st[tp.tile_prob[cur]].done))
          cur = ld_volatile(&sgl->all_done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
        s_tile = cur;
        if (cur < tp.n_tiles)
          next = ld_volatile(&sgl->all_done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
      }
      __syncthreads();
      const int tile = s_tile;
      __syncthreads();
      if (tile >= tp.n_tiles) break;
      if constexpr (sizeof(T) == 4)
        tile_matvec_body_f32<kModeSeries>(tp, tile, J, t_cm, nullptr, Vinv, partial, sm);
      else
        tile_matvec_body<T, kModeSeries>(tp, tile, J, t_cm, nullptr, Vinv, partial, sm);
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
    if (tid == 0) s_done = ld_volatile(&sgl->all_done);
    __syncthreads();
    if (s_done) break;  // every problem's rule fired at term i - 1 or earlier
    // ---- phase B: cameras (the block's first group uses the cached rows and x)
    for (int g = blockIdx.x; g < n_groups; g += G) {
      if (g == (int)blockIdx.x) {
        const bool run = c_mine && !ld_volatile(&st[c_prob].done);
        double ui[9];
        if (run) {
#pragma unroll
          for (int j = 0; j < 9; ++j) ui[j] = Uinv[(size_t)c0 * 81 + ck * 9 + j];
        }
        double y = 0.0;
        if (run) {
          for (int rb = c_r0; rb < c_r1; rb += 8) {
            T buf[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) buf[j] = (rb + j < c_r1) ? __ldcg(partial + (size_t)(rb + j) * 9 + ck) : (T)0;
#pragma unroll
            for (int j = 0; j < 8; ++j) y += (double)buf[j];
          }
        }
        if (c_cl < per_group) ys[c_cl][ck] = y;
        __syncthreads();
        double v = 0.0;
        if (run) {
#pragma unroll
          for (int j = 0; j < 9; ++j) v += ui[j] * ys[c_cl][j];
          x_reg += v;
          const T tv = (T)v;
          for (int q = c_r0; q < c_r1; ++q) t_cm[(size_t)q * 9 + ck] = tv;
        }
        __syncthreads();
        if (c_cl < per_group) {
          ys[c_cl][ck] = v * v;
          y2[c_cl][ck] = x_reg * x_reg;
        }
        __syncthreads();
        if (run && ck == 0) {
          double a = 0.0, b = 0.0;
#pragma unroll
          for (int j = 0; j < 9; ++j) {
            a += ys[c_cl][j];
            b += y2[c_cl][j];
          }
          cam_norm[2 * c0 + 0] = a;
          cam_norm[2 * c0 + 1] = b;
        }
        __syncthreads();
      } else {
        camera_body<T, kModeSeries>(tp, g * per_group, per_group, partial, nullptr, Uinv, x, t_cm,
                                    st, cam_norm, ys, y2);
      }
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (barrier_arrive(gs, G, &gen, &s_last, &s_gen)) {
      // last block: open the barrier, then every running problem's norms (camera order) and its
      // stop rule for term i (visible to every block before the next barrier)
      if (tid == 0) barrier_release(gs);
      __threadfence();
      problems_stop_rule(tp, cam_norm, st, sgl, i, eps, &s_running);
    } else if (!barrier_wait(gs, gen, timeout, &s_ok)) {
      return;
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  if (c_mine) x[(size_t)c0 * 9 + ck] = x_reg;
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
                                     const double* Uinv, double* x, T* t_cm, T* partial,
                                     double* cam_norm, SeriesState* st, SeriesGlobal* sgl,
                                     GridSync* gs, int m_max, double eps, long long timeout,
                                     long long* trace, cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&J, (void*)&Vinv, (void*)&Uinv, (void*)&x, (void*)&t_cm,
                  (void*)&partial, (void*)&cam_norm, (void*)&st, (void*)&sgl, (void*)&gs,
                  (void*)&m_max, (void*)&eps, (void*)&timeout, (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_persistent_kernel<T>, dim3(grid),
                                     dim3(kTileObs), args, 0, s);
}

template cudaError_t launch_series_persistent<double>(const Topology&, int, const double*, const double*, const double*, double*, double*, double*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);
template cudaError_t launch_series_persistent<float>(const Topology&, int, const float*, const float*, const double*, double*, float*, float*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);

}  // namespace poba
