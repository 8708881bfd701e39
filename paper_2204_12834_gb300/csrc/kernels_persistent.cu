// Persistent power-series kernel of libpoba (sm_103a): after the reduced right-hand side and
// x(0) (two per-term launches), one cooperative launch runs every series term and the stop
// rule of Sec. 4.3 (eqs. `S_approx`, `x_approx`, `qcriterion`).
//
// Each term is two phases separated by grid barriers:
//   phase A  every block but the last takes groups of the series schedule by ticket (largest
//            first) and runs the group body (W^T t, V^-1, W z, one partial row per group slot);
//   phase B  camera groups (spread over all blocks, static) run the camera body (U^-1, x
//            accumulation, new term rows) and store a squared-norm pair per camera;
//   barrier  the last block to arrive opens it by arriving; the grid's last block (the stop-rule
//            block, which takes no groups) waits for it, sums each running problem's camera norm
//            pairs in camera order and applies its stop rule while the others run the next
//            term's groups; every block sees the decisions before the next camera phase (a
//            stopped problem's groups and cameras are skipped, so its x stays at the term where
//            its rule fired).
// Results are bitwise equal to the per-term launches: every group and camera computes the same
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

// Grid barrier on a monotonic arrival counter: barrier n of a launch completes when the counter
// reaches (n + 1) G, so the last block to arrive opens it by its own arrival (no release step)
// and the others poll the counter.  Arrive: the block's writes are made visible (barrier, then
// a fence by the arriving thread), then one atomic.  Returns (in every thread) whether this block
// arrived last; the count that completes the barrier is stored in *target.
__device__ __forceinline__ int barrier_arrive(GridSync* gs, unsigned G, unsigned* target,
                                              int* s_last, unsigned* s_target) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&gs->arrive, 1u);
    *s_last = ticket % G == G - 1;
    *s_target = (ticket / G + 1) * G;
  }
  __syncthreads();
  *target = *s_target;
  return *s_last;
}

// Wait until the arrival count reaches `target`; false on timeout or when another block failed.
// Polls with an exponential back-off (32 ns .. 256 ns) to keep the hot word quiet.
__device__ __forceinline__ bool barrier_wait(GridSync* gs, unsigned target, long long timeout,
                                             int* s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    unsigned sleep_ns = 32;
    for (unsigned it = 0; ld_volatile(&gs->arrive) < target; ++it) {
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
      if (sleep_ns < 256) sleep_ns <<= 1;
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Phase B of a term: block b runs the rounds [block_round[b], block_round[b + 1]) of the camera
// schedule.  In a round, thread (item, k) sums component k of one chunk of slot rows; then
// thread (camera, k) adds its camera's chunk sums in chunk order, applies row k of U^-1, updates
// x and writes the new term t_cam[c] and the camera's norm pair -- the same sums in the same
// order as camera_body.  The block's first round is fixed for the whole launch: its item
// bounds, cameras and the cameras' x stay in registers (x is written back at the end), so a
// term's chain of dependent loads there is the chunk rows and the done flag.  Later rounds (a
// block has several when cameras outnumber the grid) load their indices each term; every load
// that does not depend on the chunk sums is issued at the start of the round.  Shared scratch
// (doubles): pc[kRoundItems][9], ys[kRoundItems][9], y2[kRoundItems][9].
constexpr int kCamScratchBytes = 3 * kRoundItems * 9 * 8;

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Row k of camera c's U^-1 (read-only during the launch) toward L1 ahead of its use.
__device__ __forceinline__ void prefetch_uinv_row(const double* __restrict__ Uinv, int c, int k) {
  const double* r = Uinv + (size_t)c * 81 + k * 9;
  prefetch_l1(r);
  prefetch_l1(r + 8);
}

struct RoundCache {  // in shared memory
  int rd, nc, ni;                 // the block's first round (rd = -1: none), its cameras, items
  int q[kRoundItems][2];          // item rows
  int cam[kRoundItems][4];        // camera, its items (round-relative), problem
  double x[kRoundItems][9];       // the cameras' x
  int done[kRoundItems];          // the current round's cameras: their problem's done flag
};

__device__ __forceinline__ void round_cache(const Topology& tp, const CamRounds& cr,
                                            const double* __restrict__ x, RoundCache& rc,
                                            int n_rows) {
  const int it = threadIdx.x / 9, k = threadIdx.x - it * 9;
  const int rd = cr.block_round[blockIdx.x] < cr.block_round[blockIdx.x + 1]
                     ? cr.block_round[blockIdx.x] : -1;
  if (threadIdx.x == 0) rc.rd = rd;
  if (rd >= 0) {
    const int c0 = cr.round_cam[rd], i0 = cr.round_item[rd];
    const int nc = cr.round_cam[rd + 1] - c0, ni = cr.round_item[rd + 1] - i0;
    if (threadIdx.x == 0) {
      rc.nc = nc;
      rc.ni = ni;
    }
    if (it < ni && k < 2) {
      int q = cr.item_q[2 * (i0 + it) + k];
      POBA_CHK(tp.chk, q, n_rows + 1, kChkCamRows);
      rc.q[it][k] = q;
    }
    if (it < nc) {
      const int c = c0 + it;
      if (k == 0) rc.cam[it][0] = c;
      if (k == 1) rc.cam[it][1] = cr.cam_item[c] - i0;
      if (k == 2) rc.cam[it][2] = cr.cam_item[c + 1] - i0;
      if (k == 3) rc.cam[it][3] = tp.cam_prob[c];
      rc.x[it][k] = x[(size_t)c * 9 + k];
    }
  }
  __syncthreads();
}

// Combination, U^-1 and norms of one round (after the chunk sums are in pc).  The round's
// cameras are c_first .. c_first + nc - 1 with their done flags in done[]; the norm pairs are
// summed by the block's first 2 nc threads (a thread per pair entry), so that only the warps
// holding them issue those FP64 adds.
template <typename T>
__device__ __forceinline__ double round_finish(bool cam, bool run, int c, int ia, int ib,
                                               const double* __restrict__ Uinv, double xo,
                                               T* __restrict__ t_cam,
                                               double* __restrict__ cam_norm, double (*pc)[9],
                                               double (*ys)[9], double (*y2)[9], int c_first,
                                               int nc, const int* done) {
  const int it = threadIdx.x / 9, k = threadIdx.x - it * 9;
  double y = 0.0;
  if (run)
    for (int j = ia; j < ib; ++j) y += pc[j][k];
  if (cam) ys[it][k] = y;
  __syncthreads();
  double v = 0.0, xv = 0.0;
  if (run) {
    const double* ui = Uinv + (size_t)c * 81 + k * 9;
#pragma unroll
    for (int j = 0; j < 9; ++j) v += __ldg(ui + j) * ys[it][j];
    xv = xo + v;
    t_cam[(size_t)c * kTStride + k] = (T)v;
  }
  __syncthreads();
  if (cam) {
    ys[it][k] = v * v;
    y2[it][k] = xv * xv;
  }
  __syncthreads();
  if (threadIdx.x < 2 * nc) {
    const int cn = threadIdx.x >> 1, e = threadIdx.x & 1;
    if (!done[cn]) cam_norm[2 * (c_first + cn) + e] = norm_row_sum(e ? y2[cn] : ys[cn]);
  }
  __syncthreads();
  return run ? xv : xo;
}

template <typename T>
__device__ __forceinline__ void camera_phase(const Topology& tp, const CamRounds& cr, int n_rows,
                                             RoundCache& rc, const T* __restrict__ partial,
                                             const double* __restrict__ Uinv,
                                             double* __restrict__ x, T* __restrict__ t_cam,
                                             double* __restrict__ cam_norm,
                                             const SeriesState* st, double* scratch) {
  double (*pc)[9] = reinterpret_cast<double (*)[9]>(scratch);
  double (*ys)[9] = pc + kRoundItems;
  double (*y2)[9] = ys + kRoundItems;
  const int tid = threadIdx.x;
  const int it = tid / 9, k = tid - it * 9;
  if (rc.rd < 0) return;
  {
    // the cached first round.  The done flags are read by one warp (a lane per camera): every
    // block reads them at once, and one request per block keeps their L2 line quiet.
    const bool cam = it < rc.nc;
    int c = 0;
    if (tid < rc.nc) rc.done[tid] = ld_volatile(&st[rc.cam[tid][3]].done);
    if (cam) {
      c = rc.cam[it][0];
      prefetch_uinv_row(Uinv, c, k);
    }
    if (it < rc.ni) pc[it][k] = cam_chunk_sum(partial, rc.q[it][0], rc.q[it][1], k);
    __syncthreads();
    const bool done = cam ? rc.done[it] != 0 : true;
    const double xo = cam ? rc.x[it][k] : 0.0;
    const double xv = round_finish<T>(cam, cam && !done, c, cam ? rc.cam[it][1] : 0,
                                      cam ? rc.cam[it][2] : 0, Uinv, xo, t_cam, cam_norm, pc,
                                      ys, y2, rc.cam[0][0], rc.nc, rc.done);
    if (cam) rc.x[it][k] = xv;
  }
  for (int rd = rc.rd + 1; rd < cr.block_round[blockIdx.x + 1]; ++rd) {
    const int c0 = cr.round_cam[rd], nc = cr.round_cam[rd + 1] - c0;
    const int i0 = cr.round_item[rd], ni = cr.round_item[rd + 1] - i0;
    const int c = c0 + it;
    const bool cam = it < nc;
    double xo = 0.0;
    int ia = 0, ib = 0;
    if (tid < nc) rc.done[tid] = ld_volatile(&st[tp.cam_prob[c0 + tid]].done);
    if (cam) {
      prefetch_uinv_row(Uinv, c, k);
      xo = __ldcg(x + (size_t)c * 9 + k);
      ia = cr.cam_item[c] - i0;
      ib = cr.cam_item[c + 1] - i0;
    }
    if (it < ni) {
      int q0 = cr.item_q[2 * (i0 + it)], q1 = cr.item_q[2 * (i0 + it) + 1];
      POBA_CHK(tp.chk, q0, n_rows + 1, kChkCamRows);
      POBA_CHK(tp.chk, q1, n_rows + 1, kChkCamRows);
      pc[it][k] = cam_chunk_sum(partial, q0, q1, k);
    }
    __syncthreads();
    const bool run = cam && rc.done[it] == 0;
    const double xv = round_finish<T>(cam, run, c, ia, ib, Uinv, xo, t_cam, cam_norm, pc, ys, y2,
                                      c0, nc, rc.done);
    if (run) x[(size_t)c * 9 + k] = xv;
  }
}

// The U^-1 blocks of the cameras of this block's rounds toward L2 (one bulk prefetch per round,
// the cameras of a round being consecutive), issued when the block leaves a group phase so that
// the camera phase after the barrier finds them there: a group phase streams the Jacobians
// through L2 and evicts them otherwise.  Thread 0 only.
__device__ __forceinline__ void prefetch_round_uinv(const CamRounds& cr, const RoundCache& rc,
                                                    const double* __restrict__ Uinv) {
  if (threadIdx.x != 0 || rc.rd < 0) return;
  for (int rd = rc.rd; rd < cr.block_round[blockIdx.x + 1]; ++rd) {
    const int c0 = cr.round_cam[rd], c1 = cr.round_cam[rd + 1];
    prefetch_l2(Uinv + (size_t)c0 * 81, (size_t)(c1 - c0) * 81 * sizeof(double), false);
  }
}

// The cached first round's x back to memory (end of the launch).
__device__ __forceinline__ void round_writeback(const RoundCache& rc, double* __restrict__ x) {
  const int it = threadIdx.x / 9, k = threadIdx.x - it * 9;
  if (rc.rd >= 0 && it < rc.nc) x[(size_t)rc.cam[it][0] * 9 + k] = rc.x[it][k];
}

// The stop-rule block of a persistent launch: the grid's last block.  It takes no groups; at the
// end of each term it waits for every camera of the term, then applies every running problem's
// stop rule while the other blocks already run the next term's groups, and only then arrives
// at that term's first barrier -- so every block sees the decisions before the next camera
// phase, and the reduction of the camera norms (thousands of cameras for a large problem) is
// off the critical path.
__device__ __forceinline__ bool stop_block() { return blockIdx.x == gridDim.x - 1; }

// Barrier 2 of a term.  False: this block must leave (a wait timed out or another block
// failed).  The stop-rule block waits for the barrier and then applies the stop rule of term i;
// every other block leaves as soon as the barrier is complete.
__device__ __forceinline__ bool term_end_barrier(const Topology& tp, GridSync* gs,
                                                 const double* cam_norm, SeriesState* st,
                                                 SeriesGlobal* sgl, int i, double eps,
                                                 long long timeout, int* s_last, unsigned* s_gen,
                                                 int* s_ok, int* s_running, double* red) {
  unsigned target;
  const bool last = barrier_arrive(gs, gridDim.x, &target, s_last, s_gen);
  if (!stop_block()) return last || barrier_wait(gs, target, timeout, s_ok);
  if (!last && !barrier_wait(gs, target, timeout, s_ok)) return false;
  __threadfence();
  problems_stop_rule(tp, cam_norm, st, sgl, i, eps, s_running, red);
  return true;
}

// Barrier 1 of a term (after the group phase): the last block resets the ticket counter.
__device__ __forceinline__ bool tile_end_barrier(GridSync* gs, long long timeout, int* s_last,
                                                 unsigned* s_gen, int* s_ok) {
  unsigned target;
  if (barrier_arrive(gs, gridDim.x, &target, s_last, s_gen)) {
    // no block claims groups again before the term's second barrier, which this block reaches
    // after the reset (its arrival there publishes it)
    if (threadIdx.x == 0) atomicExch(&gs->tile_next, 0u);
    return true;
  }
  return barrier_wait(gs, target, timeout, s_ok);
}

template <typename T>
__global__ void __launch_bounds__(kChunkObs, sizeof(T) == 4 ? 4 : 3) series_persistent_kernel(
    Topology tp, SerTopo sp, CamRounds cr, const T* __restrict__ J, const T* __restrict__ Vinv,
    const double* __restrict__ Uinv, double* __restrict__ x, T* __restrict__ t_cam,
    T* __restrict__ partial, double* __restrict__ cam_norm, SeriesState* __restrict__ st,
    SeriesGlobal* __restrict__ sgl, GridSync* __restrict__ gs, int m_max, double eps,
    long long timeout, long long* __restrict__ trace) {
  extern __shared__ __align__(16) unsigned char group_smem[];
  GroupSmem<T>& sm = *reinterpret_cast<GroupSmem<T>*>(group_smem);
  __shared__ int s_group, s_last, s_ok, s_done, s_running;
  __shared__ unsigned s_gen;
  static_assert(kCamScratchBytes <= sizeof(sm.sg), "phase B scratch fits in sg");
  const int tid = threadIdx.x;
  double* scratch = reinterpret_cast<double*>(&sm.sg[0][0]);  // phase B reuses sg

  if (tid == 0) s_done = ld_volatile(&sgl->all_done);  // every x(0) = 0: nothing to do
  __syncthreads();
  if (s_done) return;
  __shared__ RoundCache rc;
  round_cache(tp, cr, x, rc, sp.n_gslots);
  const bool tracer = blockIdx.x == 0 && tid == 0 && trace != nullptr;
  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    // ---- phase A: groups by ticket (not the stop-rule block).  Once every problem has stopped
    // the remaining groups are moot; in a batch, groups of a problem that stopped are skipped.
    for (;;) {
      if (stop_block()) break;
      if (tid == 0) {
        int g = ld_volatile(&sgl->all_done) ? sp.n_groups : (int)atomicAdd(&gs->tile_next, 1u);
        while (g < sp.n_groups && ld_volatile(&st[__ldg(sp.group + 2 * g + 1).y].done))
          g = ld_volatile(&sgl->all_done) ? sp.n_groups : (int)atomicAdd(&gs->tile_next, 1u);
        s_group = g < sp.n_groups ? g : sp.n_groups;
      }
      __syncthreads();  // also: every thread is done with the previous group's shared memory
      const int g = s_group;
      if (g >= sp.n_groups) break;
      group_body<T, kModeSeries>(tp, sp, g, J, t_cam, nullptr, Vinv, partial, sm);
    }
    prefetch_round_uinv(cr, rc, Uinv);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 1] = global_ns();
    if (!tile_end_barrier(gs, timeout, &s_last, &s_gen, &s_ok)) return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 2] = global_ns();
    if (tid == 0) s_done = ld_volatile(&sgl->all_done);
    __syncthreads();
    if (s_done) break;  // every problem's rule fired at term i - 1 or earlier
    // ---- phase B: cameras
    camera_phase<T>(tp, cr, sp.n_gslots, rc, partial, Uinv, x, t_cam, cam_norm, st, scratch);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (!term_end_barrier(tp, gs, cam_norm, st, sgl, i, eps, timeout, &s_last, &s_gen, &s_ok,
                          &s_running, scratch))
      return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  round_writeback(rc, x);
}

// ---------------------------------------------------------------------------------------
// Dataflow persistent kernel (series_exec 5): the same group and camera arithmetic with no grid
// barrier.  Tickets run over (term, group) pairs -- ticket u is group u mod G of term
// u / G + 1, groups in their longest-first order -- so a block that finishes early goes on to
// the next term's groups while others still run this term's.  What a barrier ordered before
// is ordered per camera and per problem:
//   * a group of term i starts once the term i - 1 update of each of its slots' cameras is
//     published (cam_epoch[c] >= i - 1), so it reads t_{i-1} and overwrites partial rows that
//     have been consumed;
//   * after writing its partial rows a group counts them per camera (cam_cnt); the block whose
//     count completes camera c's rows of term i runs c's camera update (the camera body's sums
//     in the same order: chunk sums of the rows, U^-1, x += t, t_cam, norm pair) and publishes
//     cam_epoch[c] = i;
//   * a term-i camera update waits for the problem's term i - 1 stop decision (prob_dec) and
//     leaves x alone if the rule fired there, so x stays at the term where the rule fired;
//   * the block whose update completes a problem's cameras of term i (pcnt, by term parity)
//     applies the problem's stop rule for term i (the same norm sums as every other form, from
//     the term's norm-pair buffer: cam_norm for even terms, cam_norm_b for odd ones) and
//     publishes prob_dec = i.
// Every wait depends only on work of earlier tickets, which blocks of this co-resident grid hold,
// so the kernel cannot deadlock.  Waits are bounded as in the barrier forms (error flag).
// The trace records, for block 0's first group of each term: its claim, the end of its group
// body, the end of its slot counting, the end of its camera updates and the end of its step.

// Wait until *flag >= want or the problem is done (*done != 0), bounded.  1: the flag is set,
// 0: the problem's rule has fired (the waiting work belongs to a term past its last one and is
// moot), -1: the wait timed out or another block failed.
__device__ __forceinline__ int flow_wait(const int* flag, int want, const int* done, GridSync* gs,
                                         long long timeout) {
  const long long t0 = clock64();
  unsigned sleep_ns = 32;
  for (unsigned it = 0;; ++it) {
    if (ld_volatile(flag) >= want) {
      __threadfence();
      return 1;
    }
    if (ld_volatile(done)) {
      __threadfence();
      return 0;
    }
    if (clock64() - t0 > timeout) {
      atomicExch(&gs->error, 1);
      return -1;
    }
    if ((it & 15u) == 15u && ld_volatile(&gs->error)) return -1;
    __nanosleep(sleep_ns);
    if (sleep_ns < 256) sleep_ns <<= 1;
  }
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// A relaxed store; after one __threadfence it publishes like a release store, so a run of flags
// behind one fence costs one fence rather than one per flag (a release store is a fence and a
// store: 28 of them in a row cost microseconds).
__device__ __forceinline__ void st_relaxed(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Camera updates of term i for the cameras own[0 .. n_own) (every thread of the block): 28
// cameras at a time, thread (camera, k) as in camera_body; each pass publishes its cameras'
// epochs.  norm_out: the term's norm pairs.
template <typename T>
__device__ __forceinline__ void flow_cameras(const Topology& tp, const SerTopo& sp, const int* own,
                                             int n_own, int i,
                                             int* cam_epoch, const T* __restrict__ partial,
                                             const double* __restrict__ Uinv,
                                             double* __restrict__ x, T* __restrict__ t_cam,
                                             double* __restrict__ norm_out, double* scratch) {
  double (*ys)[9] = reinterpret_cast<double (*)[9]>(scratch);
  double (*y2)[9] = ys + kRoundItems;
  const int cl = threadIdx.x / 9, k = threadIdx.x - 9 * cl;
  for (int base = 0; base < n_own; base += kRoundItems) {
    const bool cam = cl < kRoundItems && base + cl < n_own;
    int c = 0;
    double y = 0.0, xo = 0.0;
    if (cam) {
      c = own[base + cl];
      prefetch_uinv_row(Uinv, c, k);
      xo = __ldcg(x + (size_t)c * 9 + k);
      int r0 = __ldg(sp.cam_ptr + c), r1 = __ldg(sp.cam_ptr + c + 1);
      POBA_CHK(tp.chk, r0, sp.n_gslots + 1, kChkCamRows);
      POBA_CHK(tp.chk, r1, sp.n_gslots + 1, kChkCamRows);
      const int C = cam_chunk_rows(r1 - r0);
      for (int q0 = r0; q0 < r1; q0 += C) y += cam_chunk_sum(partial, q0, min(q0 + C, r1), k);
      ys[cl][k] = y;
    }
    __syncthreads();
    double v = 0.0, xv = 0.0;
    if (cam) {
      const double* ui = Uinv + (size_t)c * 81 + k * 9;
#pragma unroll
      for (int j = 0; j < 9; ++j) v += __ldg(ui + j) * ys[cl][j];
      xv = xo + v;
      x[(size_t)c * 9 + k] = xv;
      t_cam[(size_t)c * kTStride + k] = (T)v;
    }
    __syncthreads();
    if (cam) {
      ys[cl][k] = v * v;
      y2[cl][k] = xv * xv;
    }
    __syncthreads();
    const int nb = min(kRoundItems, n_own - base);
    if (threadIdx.x < 2 * nb) {
      const int cn = threadIdx.x >> 1, e = threadIdx.x & 1;
      norm_out[2 * own[base + cn] + e] = norm_row_sum(e ? y2[cn] : ys[cn]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      for (int j = base; j < n_own && j < base + kRoundItems; ++j) st_relaxed(cam_epoch + own[j], i);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kChunkObs, sizeof(T) == 4 ? 4 : 3) series_dataflow_kernel(
    Topology tp, SerTopo sp, FlowState fs, const T* __restrict__ J, const T* __restrict__ Vinv,
    const double* __restrict__ Uinv, double* __restrict__ x, T* __restrict__ t_cam,
    T* __restrict__ partial, double* __restrict__ cam_norm, SeriesState* __restrict__ st,
    SeriesGlobal* __restrict__ sgl, GridSync* __restrict__ gs, int m_max, double eps,
    long long timeout, long long* __restrict__ trace) {
  extern __shared__ __align__(16) unsigned char group_smem[];
  GroupSmem<T>& sm = *reinterpret_cast<GroupSmem<T>*>(group_smem);
  __shared__ int s_ticket, s_n_own, s_run, s_last;
  __shared__ int s_own[kGroupSlots];
  static_assert(2 * kRoundItems * 9 * 8 <= sizeof(sm.sg) && 2 * kNormLanes * 8 <= sizeof(sm.sg),
                "camera and stop-rule scratch fit in sg");
  const int tid = threadIdx.x;
  double* scratch = reinterpret_cast<double*>(&sm.sg[0][0]);
  const unsigned G = (unsigned)sp.n_groups;
  const unsigned total = (unsigned)m_max * G;
  const bool tracer = blockIdx.x == 0 && tid == 0 && trace != nullptr;
  int traced = 0;  // last term block 0 has traced
  for (;;) {
    // ---- claim the next ticket of a problem that is still running
    if (tid == 0) {
      int t = -1;
      while (!ld_volatile(&sgl->all_done) && !ld_volatile(&gs->error)) {
        const unsigned u = atomicAdd(&gs->tile_next, 1u);
        if (u >= total) break;
        // a problem decided done at an earlier term has no more groups to run (no group of a
        // term at or before its last decision can still be unclaimed)
        if (ld_volatile(&st[__ldg(sp.group + 2 * (u % G) + 1).y].done)) continue;
        t = (int)u;
        break;
      }
      s_ticket = t;
    }
    __syncthreads();
    const int t = s_ticket;
    if (t < 0) break;
    const int i = t / (int)G + 1, g = t % (int)G;
    const bool tr = tracer && i > traced && i <= kTraceTerms;
    if (tr) trace[(i - 1) * kTracePoints + 0] = global_ns();
    const int4 gd = __ldg(sp.group + 2 * g);
    const int s0 = gd.z, ns = gd.w, p = __ldg(sp.group + 2 * g + 1).y;
    // ---- the term i - 1 updates of the group's cameras (or the problem's rule has fired:
    // then the group is moot)
    int w = 1;
    if (i > 1 && tid < ns)
      w = flow_wait(fs.cam_epoch + __ldg(sp.gslot_cam + s0 + tid), i - 1, &st[p].done, gs, timeout);
    if (__syncthreads_or(w < 0)) return;
    if (__syncthreads_or(w == 0)) continue;  // (the claim barrier follows)
    group_body<T, kModeSeries>(tp, sp, g, J, t_cam, nullptr, Vinv, partial, sm);
    if (tr) trace[(i - 1) * kTracePoints + 1] = global_ns();
    // ---- count the group's rows per camera; the last one of a camera's term owns its update
    if (tid == 0) s_n_own = 0;
    __syncthreads();  // also: every partial row of the group is written
    if (tid < ns) {
      const int c = __ldg(sp.gslot_cam + s0 + tid);
      const unsigned rows = (unsigned)(__ldg(sp.cam_ptr + c + 1) - __ldg(sp.cam_ptr + c));
      __threadfence();
      const unsigned cnt = atomicAdd(fs.cam_cnt + c, 1u) + 1u;
      if (cnt == (unsigned)i * rows) {
        __threadfence();
        s_own[atomicAdd(&s_n_own, 1)] = c;
      }
    }
    __syncthreads();
    if (tr) trace[(i - 1) * kTracePoints + 2] = trace[(i - 1) * kTracePoints + 3] = global_ns();
    const int n_own = s_n_own;
    if (n_own > 0) {
      // the problem's term i - 1 decision: x moves only while the problem runs
      if (tid == 0) {
        const int r = flow_wait(fs.prob_dec + p, i - 1, &st[p].done, gs, timeout);
        s_run = r < 0 ? -1 : (r == 0 || ld_volatile(&st[p].done)) ? 0 : 1;
      }
      __syncthreads();
      const int run = s_run;
      if (run < 0) return;
      double* norm_out = (i & 1) ? fs.cam_norm_b : cam_norm;
      if (run) {
        flow_cameras<T>(tp, sp, s_own, n_own, i, fs.cam_epoch, partial, Uinv, x, t_cam, norm_out,
                        scratch);
      } else if (tid == 0) {
        __threadfence();
        for (int j = 0; j < n_own; ++j) st_relaxed(fs.cam_epoch + s_own[j], i);
      }
      if (tid == 0) {
        int last = 0;
        if (run) {
          const unsigned want = (unsigned)((i + 1) / 2) * (unsigned)__ldg(sp.prob_ncam + p);
          last = atomicAdd(fs.pcnt + 2 * p + (i & 1), (unsigned)n_own) + (unsigned)n_own == want;
        }
        s_last = last;
        if (last) __threadfence();
      }
      if (tr) trace[(i - 1) * kTracePoints + 3] = global_ns();
      __syncthreads();
      if (s_last) {
        // this block completed problem p's cameras of term i: its stop rule (the decision of
        // term i - 1 is in place: every term-i update waited for it)
        const int c0 = tp.cam_off[p], c1 = tp.cam_off[p + 1];
        double a = 0.0, b = 0.0;
        if (c1 - c0 >= kBlockNormCams) {
          block_norm_sums(norm_out, c0, c1, scratch, a, b);
        } else if (tid < 32) {
          warp_norm_sums(norm_out, c0, c1, a, b);
        }
        if (tid == 0) {
          series_stop_rule(&st[p], i, a, b, eps);
          const bool stop = st[p].done != 0;
          __threadfence();
          if (stop && atomicSub(&sgl->n_running, 1) == 1) atomicExch(&sgl->all_done, 1);
          st_release(fs.prob_dec + p, i);
        }
      }
    }
    if (tr) {
      trace[(i - 1) * kTracePoints + 4] = global_ns();
      traced = i;
    }
    __syncthreads();  // every thread is done with this group's shared memory
  }
}

template <typename T>
int dataflow_blocks_per_sm() {
  if (cudaFuncSetAttribute(series_dataflow_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(GroupSmem<T>)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_dataflow_kernel<T>, kChunkObs,
                                                    sizeof(GroupSmem<T>)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename T>
cudaError_t launch_series_dataflow(const Topology& tp, const SerTopo& sp, const FlowState& fs,
                                   int grid, const T* J, const T* Vinv, const double* Uinv,
                                   double* x, T* t_cam, T* partial, double* cam_norm,
                                   SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                   double eps, long long timeout, long long* trace,
                                   cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&sp, (void*)&fs, (void*)&J, (void*)&Vinv, (void*)&Uinv,
                  (void*)&x, (void*)&t_cam, (void*)&partial, (void*)&cam_norm, (void*)&st,
                  (void*)&sgl, (void*)&gs, (void*)&m_max, (void*)&eps, (void*)&timeout,
                  (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_dataflow_kernel<T>, dim3(grid),
                                     dim3(kChunkObs), args, sizeof(GroupSmem<T>), s);
}

template int dataflow_blocks_per_sm<double>();
template int dataflow_blocks_per_sm<float>();
template cudaError_t launch_series_dataflow<double>(const Topology&, const SerTopo&, const FlowState&, int, const double*, const double*, const double*, double*, double*, double*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);
template cudaError_t launch_series_dataflow<float>(const Topology&, const SerTopo&, const FlowState&, int, const float*, const float*, const double*, double*, float*, float*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);

// ---------------------------------------------------------------------------------------
// FP32-bulk persistent kernel with staged chunks (series_exec 4).  The arithmetic is the group
// body's (chunk_f32_core: the same sums in the same order as every other form); what changes is
// how a chunk's inputs reach the threads.  One thread copies each chunk -- its six Jacobian
// plane groups, its record and its landmarks' V^-1 rows -- into shared memory with bulk
// asynchronous copies (cp.async.bulk, completion counted on an mbarrier), one chunk ahead: the
// copies of chunk k + 1 go out once every thread holds chunk k's inputs in registers (the first
// barrier of chunk k), so they arrive while chunk k computes.  The next group is claimed one
// group ahead, so the stream of copies runs across group boundaries.  Every mbarrier wait is
// bounded (kCopyWaitCycles); a block whose wait gives up leaves with the error flag set after
// waiting (bounded) for the copy it started; the other blocks leave at their next grid barrier.
struct __align__(16) F32Stage {
  float4 J[6][kChunkObs];                    // plane groups 0..5 of the chunk's observations
  alignas(16) uint8_t rec[kChunkRecMax];     // the chunk record
  alignas(16) float vi[kChunkObs * 6 + 8];   // V^-1 rows of its landmarks (range rounded out)
  unsigned long long mbar;
};
static_assert(offsetof(F32Stage, rec) % 16 == 0 && offsetof(F32Stage, vi) % 16 == 0 &&
                  offsetof(F32Stage, mbar) % 8 == 0 && kChunkRecMax % 16 == 0,
              "bulk-copy destinations must be 16-byte aligned");

struct StagedSmem {
  GroupSmem<float> g;
  F32Stage s;
};

// Bound on a wait for this block's own copies (about 4 s at 2 GHz).
constexpr long long kCopyWaitCycles = 1LL << 33;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arm(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false after `timeout` cycles.
__device__ __forceinline__ bool mbar_wait(unsigned long long* mb, unsigned parity,
                                          long long timeout) {
  const long long t0 = clock64();
  while (!mbar_try(mb, parity))
    if (clock64() - t0 > timeout) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(mb))
      : "memory");
}

// One thread: bulk copies of the chunk with descriptor {d0, d1} into the stage (the stage's
// previous contents have been read by every thread: the caller is past a block barrier that
// follows the last read).
__device__ __forceinline__ void f32_issue(F32Stage& S, const SerTopo& sp, const int4& d0,
                                          const int4& d1, const float* __restrict__ J, size_t pad,
                                          const float* __restrict__ Vinv) {
  const int o0 = d0.x, n = d0.y, L0 = d0.z, nl = d0.w;
  const unsigned jb = (unsigned)n * 16u;
  const unsigned rb = (unsigned)chunk_rec_layout(n, nl, d1.x).bytes;
  const size_t v0 = ((size_t)L0 * 6) & ~(size_t)3, v1 = ((size_t)(L0 + nl) * 6 + 3) & ~(size_t)3;
  const unsigned vb = (unsigned)(v1 - v0) * 4u;
  // the stage was last read through the generic proxy; order those reads before the copies
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arm(&S.mbar, 6u * jb + rb + vb);
  const float4* G = reinterpret_cast<const float4*>(J);
#pragma unroll
  for (int q = 0; q < 6; ++q) bulk_g2s(&S.J[q][0], G + (size_t)q * pad + o0, jb, &S.mbar);
  bulk_g2s(S.rec, sp.rec + (size_t)d1.y * 16, rb, &S.mbar);
  bulk_g2s(S.vi, Vinv + v0, vb, &S.mbar);
}

// The inputs of an active thread from the staged chunk.
__device__ __forceinline__ void f32_load_staged(const Topology& tp, const F32Stage& S,
                                                const int4& d0, const ChunkRecLayout& L, F32Obs& x,
                                                int gns) {
  const int tid = threadIdx.x;
  float all[24];
#pragma unroll
  for (int q = 0; q < 6; ++q) unpack16(S.J[q][tid], all + 4 * q);
#pragma unroll
  for (int p = 0; p < 18; ++p) x.jp[p] = all[p];
#pragma unroll
  for (int p = 0; p < 6; ++p) x.jl[p] = all[18 + p];
  x.code = chk_code(tp, reinterpret_cast<const uint32_t*>(S.rec + L.code)[tid], d0.y, d0.w, gns);
  const int lm = (int)(x.code >> 16) & 0xff;
  const uint16_t* sseg = reinterpret_cast<const uint16_t*>(S.rec + L.sseg);
  x.a = sseg[lm];
  x.b = sseg[lm + 1];
  chk_seg(tp, x.a, x.b, d0.y);
  f32_vinv(x, S.vi + (((size_t)d0.z * 6) & 3) + (size_t)lm * 6);
}

// The issuing thread of the staged kernel: the first lane of the last warp, whose share of a
// chunk's slot sums is the smallest (chunk slots are ordered longest first).
constexpr int kIssuer = kChunkObs - 32;

// Ticket of the next group whose problem still runs (n_groups: none).
__device__ __forceinline__ int claim_group(const SerTopo& sp, const SeriesState* st,
                                           const SeriesGlobal* sgl, GridSync* gs) {
  int g = ld_volatile(&sgl->all_done) ? sp.n_groups : (int)atomicAdd(&gs->tile_next, 1u);
  while (g < sp.n_groups && ld_volatile(&st[__ldg(sp.group + 2 * g + 1).y].done))
    g = ld_volatile(&sgl->all_done) ? sp.n_groups : (int)atomicAdd(&gs->tile_next, 1u);
  return g < sp.n_groups ? g : sp.n_groups;
}

// Phase A of one term with staged chunks.  Returns false (in every thread) if a copy wait gave
// up; thread 0 has then waited (bounded) for the copy it had started.
__device__ __forceinline__ bool groups_staged(const Topology& tp, const SerTopo& sp,
                                              const float* __restrict__ J,
                                              const float* __restrict__ Vinv,
                                              const float* __restrict__ t_cam,
                                              float* __restrict__ partial, StagedSmem& sm,
                                              unsigned& par, const SeriesState* st,
                                              const SeriesGlobal* sgl, GridSync* gs,
                                              int* s_group) {
  const int tid = threadIdx.x;
  const size_t pad = (size_t)tp.n_obs_pad;
  // The issuing thread walks the block's stream of chunks one chunk ahead of the copies in
  // flight: pend is the next chunk to copy (-1: none), with its descriptor already loaded so that
  // issuing waits on no load, and pend_end the end of its group's chunk range.  When the walk
  // leaves a group it claims the next one (a ticket taken about a chunk before the group
  // starts, so that blocks reserve no more work than they are about to run) and queues it for
  // the group loop (at most two groups ahead of the current one).
  int pend = -1, pend_end = 0, qa = sp.n_groups, qb = sp.n_groups;
  int4 pd0 = make_int4(0, 0, 0, 0), pd1 = pd0;
  auto fetch = [&](int c) {
    pend = c;
    if (c >= 0) {
      pd0 = __ldg(sp.chunk + 2 * c);
      pd1 = __ldg(sp.chunk + 2 * c + 1);
    }
  };
  // the chunk after pend in the stream
  auto advance = [&]() {
    if (pend + 1 < pend_end) {
      fetch(pend + 1);
      return;
    }
    const int g2 = claim_group(sp, st, sgl, gs);
    if (g2 >= sp.n_groups) {
      fetch(-1);
      return;
    }
    if (qa >= sp.n_groups) qa = g2;
    else qb = g2;
    const int4 ge = __ldg(sp.group + 2 * g2);
    pend_end = ge.x + ge.y;
    fetch(ge.x);
  };
  if (tid == kIssuer) {
    const int g = claim_group(sp, st, sgl, gs);
    *s_group = g;
    if (g < sp.n_groups) {
      const int4 gd = __ldg(sp.group + 2 * g);
      pend_end = gd.x + gd.y;
      fetch(gd.x);
      f32_issue(sm.s, sp, pd0, pd1, J, pad, Vinv);
      advance();
    }
  }
  __syncthreads();
  int g = *s_group;
  while (g < sp.n_groups) {
    const int4 gd = __ldg(sp.group + 2 * g);
    const int c0 = gd.x, nc = gd.y, s0 = gd.z, ns_g = gd.w;
    for (int i = tid; i < ns_g * 3; i += kChunkObs) {
      const int s = i / 3, q = i - 3 * s;
      sm.g.acc[s][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      int cam = __ldg(sp.gslot_cam + s0 + s);
      POBA_CHK(tp.chk, cam, tp.n_cams, kChkSerCam);
      sm.g.tc[s][q] = __ldcg(reinterpret_cast<const float4*>(t_cam + (size_t)cam * kTStride) + q);
    }
    __syncthreads();
    for (int c = c0; c < c0 + nc; ++c) {
      const unsigned wait_par = par;
      const bool ok = mbar_wait(&sm.s.mbar, wait_par, kCopyWaitCycles);
      par ^= 1u;
      const int4 d0 = __ldg(sp.chunk + 2 * c), d1 = __ldg(sp.chunk + 2 * c + 1);
      const int n = d0.y, ns = d1.x;
      const ChunkRecLayout L = chunk_rec_layout(n, d0.w, ns);
      const bool active = tid < n;
      F32Obs x;
      const int gns = ns_g;
      if (active) f32_load_staged(tp, sm.s, d0, L, x, gns);
      else f32_clear(x);
      x.cl = tid < ns ? chk_clist(tp, reinterpret_cast<const uint32_t*>(sm.s.rec + L.clist)[tid], n,
                                  gns)
                      : 0u;
      bool issued = false;
      const bool all_ok = chunk_f32_core<kModeSeries>(x, active, n, ns, c & 1, 0.f, 0.f, 0.f, ok,
                                                      sm.g, [&] {
        if (tid == kIssuer && pend >= 0) {
          f32_issue(sm.s, sp, pd0, pd1, J, pad, Vinv);
          issued = true;
        }
      });
      if (!all_ok) {
        if (tid == kIssuer) mbar_wait(&sm.s.mbar, wait_par, kCopyWaitCycles);
        return false;
      }
      // the walk's next step (descriptor loads, at a group's end a ticket) after the chunk's
      // slot sums, where the issuing warp (the last, with the shortest slots) has slack
      if (issued) advance();
    }
    __syncthreads();
    for (int i = tid; i < ns_g * 9; i += kChunkObs) {
      const int s = i / 9, k = i - 9 * s;
      int row = __ldg(sp.gslot_row + s0 + s);
      POBA_CHK(tp.chk, row, sp.n_gslots, kChkSerRow);
      partial[(size_t)row * 9 + k] = reinterpret_cast<const float*>(sm.g.acc[s])[k];
    }
    if (tid == kIssuer) {
      // the next group: the oldest one the walk claimed (its first chunk is in flight)
      *s_group = qa;
      qa = qb;
      qb = sp.n_groups;
    }
    __syncthreads();
    g = *s_group;
  }
  return true;
}

__global__ void __launch_bounds__(kChunkObs, 3) series_staged_kernel(
    Topology tp, SerTopo sp, CamRounds cr, const float* __restrict__ J,
    const float* __restrict__ Vinv, const double* __restrict__ Uinv, double* __restrict__ x,
    float* __restrict__ t_cam, float* __restrict__ partial, double* __restrict__ cam_norm,
    SeriesState* __restrict__ st, SeriesGlobal* __restrict__ sgl, GridSync* __restrict__ gs,
    int m_max, double eps, long long timeout, long long* __restrict__ trace) {
  extern __shared__ __align__(16) unsigned char staged_smem[];
  StagedSmem& sm = *reinterpret_cast<StagedSmem*>(staged_smem);
  __shared__ int s_group, s_last, s_ok, s_done, s_running;
  __shared__ unsigned s_gen;
  static_assert(kCamScratchBytes <= sizeof(sm.g.sg), "phase B scratch fits in sg");
  const int tid = threadIdx.x;
  double* scratch = reinterpret_cast<double*>(&sm.g.sg[0][0]);  // phase B reuses sg

  if (tid == 0) {
    s_done = ld_volatile(&sgl->all_done);  // every x(0) = 0: nothing to do
    mbar_init(&sm.s.mbar);
  }
  __syncthreads();
  if (s_done) return;
  __shared__ RoundCache rc;
  round_cache(tp, cr, x, rc, sp.n_gslots);
  unsigned par = 0u;  // parity of the stage's next mbarrier phase
  const bool tracer = blockIdx.x == 0 && tid == 0 && trace != nullptr;
  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    if (!stop_block() && !groups_staged(tp, sp, J, Vinv, t_cam, partial, sm, par, st, sgl, gs, &s_group)) {
      if (tid == 0) atomicExch(&gs->error, 1);
      return;
    }
    prefetch_round_uinv(cr, rc, Uinv);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 1] = global_ns();
    if (!tile_end_barrier(gs, timeout, &s_last, &s_gen, &s_ok)) return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 2] = global_ns();
    if (tid == 0) s_done = ld_volatile(&sgl->all_done);
    __syncthreads();
    if (s_done) break;
    camera_phase<float>(tp, cr, sp.n_gslots, rc, partial, Uinv, x, t_cam, cam_norm, st, scratch);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (!term_end_barrier(tp, gs, cam_norm, st, sgl, i, eps, timeout, &s_last, &s_gen, &s_ok,
                          &s_running, scratch))
      return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  round_writeback(rc, x);
}

int staged_blocks_per_sm() {
  if (cudaFuncSetAttribute(series_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(StagedSmem)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_staged_kernel, kChunkObs,
                                                    sizeof(StagedSmem)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_series_staged(const Topology& tp, const SerTopo& sp, const CamRounds& cr,
                                 int grid, const float* J, const float* Vinv, const double* Uinv,
                                 double* x, float* t_cam, float* partial, double* cam_norm,
                                 SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                 double eps, long long timeout, long long* trace,
                                 cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&sp, (void*)&cr, (void*)&J, (void*)&Vinv, (void*)&Uinv,
                  (void*)&x, (void*)&t_cam, (void*)&partial, (void*)&cam_norm, (void*)&st,
                  (void*)&sgl, (void*)&gs, (void*)&m_max, (void*)&eps, (void*)&timeout,
                  (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_staged_kernel, dim3(grid),
                                     dim3(kChunkObs), args, sizeof(StagedSmem), s);
}

template <typename T>
int blocks_per_sm_of() {
  if (cudaFuncSetAttribute(series_persistent_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(GroupSmem<T>)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_kernel<T>, kChunkObs,
                                                    sizeof(GroupSmem<T>)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

int persistent_blocks_per_sm(bool f32) {
  return f32 ? blocks_per_sm_of<float>() : blocks_per_sm_of<double>();
}

template <typename T>
cudaError_t launch_series_persistent(const Topology& tp, const SerTopo& sp, const CamRounds& cr,
                                     int grid, const T* J, const T* Vinv, const double* Uinv,
                                     double* x, T* t_cam, T* partial, double* cam_norm,
                                     SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                     double eps, long long timeout, long long* trace,
                                     cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&sp, (void*)&cr, (void*)&J, (void*)&Vinv, (void*)&Uinv,
                  (void*)&x, (void*)&t_cam, (void*)&partial, (void*)&cam_norm, (void*)&st,
                  (void*)&sgl, (void*)&gs, (void*)&m_max, (void*)&eps, (void*)&timeout,
                  (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_persistent_kernel<T>, dim3(grid),
                                     dim3(kChunkObs), args, sizeof(GroupSmem<T>), s);
}

template cudaError_t launch_series_persistent<double>(const Topology&, const SerTopo&, const CamRounds&, int, const double*, const double*, const double*, double*, double*, double*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);
template cudaError_t launch_series_persistent<float>(const Topology&, const SerTopo&, const CamRounds&, int, const float*, const float*, const double*, double*, float*, float*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);

}  // namespace poba
