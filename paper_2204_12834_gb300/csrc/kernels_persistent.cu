// Persistent power-series kernel of libpoba (sm_103a): after the reduced right-hand side and
// x(0) (two per-term launches), one cooperative launch runs every series term and the stop
// rule of Sec. 4.3 (eqs. `S_approx`, `x_approx`, `qcriterion`).
//
// Each term is two phases separated by grid barriers:
//   phase A  every block pulls tiles from a shared counter and runs the tile body (W^T t,
//            V^-1, W z) -- dynamic scheduling, so no wave tail;
//   phase B  camera groups (spread over all blocks, static) run the camera body (U^-1, x
//            accumulation, new term rows) and store a squared-norm pair per camera;
//   barrier  the last block to arrive opens it by arriving, then sums each running problem's
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
};

__device__ __forceinline__ void round_cache(const Topology& tp, const CamRounds& cr,
                                            const double* __restrict__ x, RoundCache& rc) {
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
    if (it < ni && k < 2) rc.q[it][k] = cr.item_q[2 * (i0 + it) + k];
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

// Combination, U^-1 and norms of one round (after the chunk sums are in pc).
template <typename T>
__device__ __forceinline__ double round_finish(bool cam, bool run, int c, int ia, int ib,
                                               const double* __restrict__ Uinv, double xo,
                                               T* __restrict__ t_cam,
                                               double* __restrict__ cam_norm, double (*pc)[9],
                                               double (*ys)[9], double (*y2)[9]) {
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
  if (run && k == 0) {
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      a += ys[it][j];
      b += y2[it][j];
    }
    cam_norm[2 * c + 0] = a;
    cam_norm[2 * c + 1] = b;
  }
  __syncthreads();
  return run ? xv : xo;
}

template <typename T>
__device__ __forceinline__ void camera_phase(const Topology& tp, const CamRounds& cr,
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
    // the cached first round
    const bool cam = it < rc.nc;
    int c = 0, done = 1;
    if (cam) {
      c = rc.cam[it][0];
      prefetch_uinv_row(Uinv, c, k);
      done = ld_volatile(&st[rc.cam[it][3]].done);
    }
    if (it < rc.ni) pc[it][k] = cam_chunk_sum(partial, rc.q[it][0], rc.q[it][1], k);
    __syncthreads();
    const double xo = cam ? rc.x[it][k] : 0.0;
    const double xv = round_finish<T>(cam, cam && !done, c, cam ? rc.cam[it][1] : 0,
                                      cam ? rc.cam[it][2] : 0, Uinv, xo, t_cam, cam_norm, pc,
                                      ys, y2);
    if (cam) rc.x[it][k] = xv;
  }
  for (int rd = rc.rd + 1; rd < cr.block_round[blockIdx.x + 1]; ++rd) {
    const int c0 = cr.round_cam[rd], nc = cr.round_cam[rd + 1] - c0;
    const int i0 = cr.round_item[rd], ni = cr.round_item[rd + 1] - i0;
    const int c = c0 + it;
    const bool cam = it < nc;
    double xo = 0.0;
    int ia = 0, ib = 0, done = 1;
    if (cam) {
      prefetch_uinv_row(Uinv, c, k);
      xo = __ldcg(x + (size_t)c * 9 + k);
      ia = cr.cam_item[c] - i0;
      ib = cr.cam_item[c + 1] - i0;
      done = ld_volatile(&st[tp.cam_prob[c]].done);
    }
    if (it < ni) {
      const int q0 = cr.item_q[2 * (i0 + it)], q1 = cr.item_q[2 * (i0 + it) + 1];
      pc[it][k] = cam_chunk_sum(partial, q0, q1, k);
    }
    __syncthreads();
    const bool run = cam && !done;
    const double xv = round_finish<T>(cam, run, c, ia, ib, Uinv, xo, t_cam, cam_norm, pc, ys, y2);
    if (run) x[(size_t)c * 9 + k] = xv;
  }
}

// The cached first round's x back to memory (end of the launch).
__device__ __forceinline__ void round_writeback(const RoundCache& rc, double* __restrict__ x) {
  const int it = threadIdx.x / 9, k = threadIdx.x - it * 9;
  if (rc.rd >= 0 && it < rc.nc) x[(size_t)rc.cam[it][0] * 9 + k] = rc.x[it][k];
}

// Barrier 2 of a term: the last block opens it, then applies every running problem's stop rule
// for term i (visible to every block before the next barrier).  False: this block must leave
// (a wait timed out or another block failed).
__device__ __forceinline__ bool term_end_barrier(const Topology& tp, GridSync* gs,
                                                 const double* cam_norm, SeriesState* st,
                                                 SeriesGlobal* sgl, int i, double eps,
                                                 long long timeout, int* s_last, unsigned* s_gen,
                                                 int* s_ok, int* s_running) {
  unsigned target;
  if (barrier_arrive(gs, gridDim.x, &target, s_last, s_gen)) {
    __threadfence();
    problems_stop_rule(tp, cam_norm, st, sgl, i, eps, s_running);
    return true;
  }
  return barrier_wait(gs, target, timeout, s_ok);
}

// Barrier 1 of a term (after the tile phase): the last block resets the tile counter.
__device__ __forceinline__ bool tile_end_barrier(GridSync* gs, long long timeout, int* s_last,
                                                 unsigned* s_gen, int* s_ok) {
  unsigned target;
  if (barrier_arrive(gs, gridDim.x, &target, s_last, s_gen)) {
    // no block claims tiles again before the term's second barrier, which this block reaches
    // after the reset (its arrival there publishes it)
    if (threadIdx.x == 0) atomicExch(&gs->tile_next, 0u);
    return true;
  }
  return barrier_wait(gs, target, timeout, s_ok);
}

template <typename T>
__global__ void __launch_bounds__(kTileObs, sizeof(T) == 4 ? 4 : 3) series_persistent_kernel(
    Topology tp, CamRounds cr, const T* __restrict__ J, const T* __restrict__ Vinv,
    const double* __restrict__ Uinv, double* __restrict__ x, T* __restrict__ t_cam,
    T* __restrict__ partial, double* __restrict__ cam_norm, SeriesState* __restrict__ st,
    SeriesGlobal* __restrict__ sgl, GridSync* __restrict__ gs, int m_max, double eps,
    long long timeout, long long* __restrict__ trace) {
  __shared__ TileSmem<T> sm;
  __shared__ int s_tile, s_last, s_ok, s_done, s_running;
  __shared__ unsigned s_gen;
  static_assert(kCamScratchBytes <= sizeof(sm.sg), "phase B scratch fits in sg");
  const int tid = threadIdx.x;
  double* scratch = reinterpret_cast<double*>(&sm.sg[0][0]);  // phase B reuses sg

  if (tid == 0) s_done = ld_volatile(&sgl->all_done);  // every x(0) = 0: nothing to do
  __syncthreads();
  if (s_done) return;
  __shared__ RoundCache rc;
  round_cache(tp, cr, x, rc);
  const bool tracer = blockIdx.x == gridDim.x - 1 && tid == 0 && trace != nullptr;
  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    // ---- phase A: tiles.  Thread 0 claims the next ticket while the current tile is
    // processed and reads the all-stopped flag for the claim after that, so neither round trip
    // holds the block (tickets at or past n_tiles mean none).  Once every problem has stopped
    // the remaining tiles are moot (a block may still take one); in a batch, tiles of a problem
    // that stopped are skipped.
    int next = 0, stop_seen = 0;
    if (tid == 0) {
      stop_seen = ld_volatile(&sgl->all_done) || (tp.n_probs == 1 && ld_volatile(&st[0].done));
      next = stop_seen ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
    }
    for (;;) {
      if (tid == 0) {
        int cur = next < tp.n_tiles ? next : tp.n_tiles;
        if (tp.n_probs > 1) {
          while (cur < tp.n_tiles && ld_volatile(&st[tp.tile_prob[cur]].done)) {
            cur = ld_volatile(&sgl->all_done) ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
            if (cur > tp.n_tiles) cur = tp.n_tiles;
          }
        }
        s_tile = cur;
        if (cur < tp.n_tiles) next = stop_seen ? tp.n_tiles : (int)atomicAdd(&gs->tile_next, 1u);
        stop_seen = ld_volatile(&sgl->all_done);  // used by the next claim
      }
      __syncthreads();
      const int tile = s_tile;
      __syncthreads();
      if (tile >= tp.n_tiles) break;
      if constexpr (sizeof(T) == 4)
        tile_matvec_body_f32<kModeSeries>(tp, tile, J, t_cam, nullptr, Vinv, partial, sm);
      else
        tile_matvec_body<T, kModeSeries>(tp, tile, J, t_cam, nullptr, Vinv, partial, sm);
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 1] = global_ns();
    if (!tile_end_barrier(gs, timeout, &s_last, &s_gen, &s_ok)) return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 2] = global_ns();
    if (tid == 0) s_done = ld_volatile(&sgl->all_done);
    __syncthreads();
    if (s_done) break;  // every problem's rule fired at term i - 1 or earlier
    // ---- phase B: cameras
    camera_phase<T>(tp, cr, rc, partial, Uinv, x, t_cam, cam_norm, st, scratch);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (!term_end_barrier(tp, gs, cam_norm, st, sgl, i, eps, timeout, &s_last, &s_gen, &s_ok,
                          &s_running))
      return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  round_writeback(rc, x);
}

// ---------------------------------------------------------------------------------------
// FP32-bulk persistent kernel with a software-pipelined tile phase.  The tile body is the one
// of the per-term kernel (f32_tile_core: the same sums in the same order); what changes is how
// a tile's inputs reach shared memory.  A block's tiles are claimed ahead and their inputs
// arrive while earlier tiles compute:
//   descriptor    32-byte asynchronous copy, three tiles ahead;
//   index record  one bulk copy (cp.async.bulk, completion on an mbarrier), two tiles ahead;
//   Jacobians     24 bulk copies (one per plane, the tile's range rounded out to 16 bytes), one
//                 tile ahead, issued as soon as the current tile's J has moved to registers;
//   t rows, V^-1  asynchronous copies issued in the middle of the previous tile, once its
//                 index record (slot rows) has arrived.
// The tiles come from a list of descriptors (the handle's tiles, or for a batch the tiles of
// the problems taking part in the solve); any block may take any tile (one atomic ticket per
// tile).  A block that finds no tile leaves the phase with nothing in flight.  Every mbarrier
// wait is bounded (kCopyWaitCycles); a block that gives up sets the error flag, waits (bounded)
// for the copies it started, and leaves; the others leave at their next grid barrier.
constexpr int kJStage = kTileObs + 4;  // floats per staged plane: the tile range rounded out

struct __align__(16) F32Pipe {
  float sJ[24][kJStage];
  uint8_t rec[3][kTileRecMax];
  float tc[2][kTileSlots][kTStride];
  float vi[2][kTileLms][6];
  float sv[kTileObs][3];
  float sg[kTileObs][9];  // the scatter; phase B's doubles
  int4 desc[4][2];
  unsigned long long mbJ;
  unsigned long long mbR[3];
};
static_assert(offsetof(F32Pipe, rec) % 16 == 0 && offsetof(F32Pipe, tc) % 16 == 0 &&
                  offsetof(F32Pipe, vi) % 16 == 0 && offsetof(F32Pipe, sg) % 16 == 0 &&
                  offsetof(F32Pipe, sv) % 16 == 0 &&
                  offsetof(F32Pipe, desc) % 16 == 0 && offsetof(F32Pipe, mbJ) % 8 == 0,
              "bulk-copy destinations must be 16-byte aligned");
static_assert((kJStage * 4) % 16 == 0 && kTileRecMax % 16 == 0, "16-byte rows");
static_assert(kCamScratchBytes <= sizeof(float) * kTileObs * 9, "phase B scratch fits in sg");

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb)) : "memory");
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
// Bound on a wait for this block's own copies (about 4 s at 2 GHz).  Independent of the grid
// barrier limit: a copy that was started is always waited for.
constexpr long long kCopyWaitCycles = 1LL << 33;

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
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Warp 0: bulk copies of the 24 Jacobian planes of the tile {o0, n} into sJ, one plane per lane
// (lane 0 arms the barrier first).
__device__ __forceinline__ void issue_J(F32Pipe& S, const float* __restrict__ J, size_t pad,
                                        int o0, int n, int lane) {
  const int a0 = o0 & ~3, e = (o0 + n + 3) & ~3;
  const unsigned bytes = (unsigned)(e - a0) * 4u;
  if (lane == 0) mbar_arm(&S.mbJ, n > 0 ? 24u * bytes : 0u);
  __syncwarp();
  if (n > 0 && lane < 24) bulk_g2s(&S.sJ[lane][0], J + (size_t)lane * pad + a0, bytes, &S.mbJ);
}

// Thread 0: bulk copy of a tile's index record into ring slot r.
__device__ __forceinline__ void issue_rec(F32Pipe& S, const uint8_t* __restrict__ recs, int r,
                                          const int4 (&d)[2]) {
  const unsigned bytes = (unsigned)tile_rec_layout(d[0].w, d[1].y, d[0].y).bytes;
  mbar_arm(&S.mbR[r], bytes);
  bulk_g2s(&S.rec[r][0], recs + (size_t)d[1].z * 16, bytes, &S.mbR[r]);
}

__global__ void __launch_bounds__(kTileObs, 3) series_persistent_f32_kernel(
    Topology tp, CamRounds cr, const int4* __restrict__ list, const int* __restrict__ n_list_p,
    const float* __restrict__ J, const float* __restrict__ Vinv, const double* __restrict__ Uinv,
    double* __restrict__ x, float* __restrict__ t_cam, float* __restrict__ partial,
    double* __restrict__ cam_norm, SeriesState* __restrict__ st, SeriesGlobal* __restrict__ sgl,
    GridSync* __restrict__ gs, int m_max, double eps, long long timeout,
    long long* __restrict__ trace) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  F32Pipe& S = *reinterpret_cast<F32Pipe*>(dyn_smem);
  __shared__ int s_last, s_ok, s_done, s_running, s_fail;
  __shared__ int s_tk[4];  // tickets of the tiles in desc[] (>= n_list: none)
  __shared__ unsigned s_gen;
  const int tid = threadIdx.x;
  const size_t pad = (size_t)tp.n_obs_pad;
  double* scratch = reinterpret_cast<double*>(&S.sg[0][0]);  // phase B reuses sg

  if (tid == 0) {
    s_done = ld_volatile(&sgl->all_done);
    s_fail = 0;
    mbar_init(&S.mbJ);
    for (int r = 0; r < 3; ++r) mbar_init(&S.mbR[r]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s_done) return;
  const int n_list = *n_list_p;
  __shared__ RoundCache rc;
  round_cache(tp, cr, x, rc);
  unsigned parJ = 0u, parR = 0u;  // phase parity of mbJ and of mbR[0..2] (bit r)
  unsigned pend = 0u;  // armed barriers not yet waited for (bit r: mbR[r], bit 3: mbJ)
  const bool tracer = blockIdx.x == gridDim.x - 1 && tid == 0 && trace != nullptr;

  for (int i = 1; i <= m_max; ++i) {
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 0] = global_ns();
    // ---- phase A, prologue: claim three tiles, fetch their descriptors, start the first
    // two records and the first Jacobians
    int tk_next = n_list;  // thread 0: ticket claimed for the slot after the last filled one
    int stop_seen = 0;     // thread 0: the all-stopped flag as of the previous claim
    if (tid < 32) {
      if (tid == 0) {
        int t0 = n_list;
        if (!ld_volatile(&sgl->all_done)) t0 = (int)atomicAdd(&gs->tile_next, 3u);
        for (int q = 0; q < 3; ++q) {
          const int tk = t0 + q < n_list ? t0 + q : n_list;
          s_tk[q] = tk;
          if (tk < n_list) {
            cp_async16(&S.desc[q][0], list + 2 * (size_t)tk);
            cp_async16(&S.desc[q][1], list + 2 * (size_t)tk + 1);
          }
        }
        cp_async_wait_all();
        if (t0 + 2 < n_list) tk_next = (int)atomicAdd(&gs->tile_next, 1u);
        if (s_tk[0] < n_list) {
          issue_rec(S, tp.tile_rec, 0, S.desc[0]);
          pend |= 9u;
        }
        if (s_tk[1] < n_list) {
          issue_rec(S, tp.tile_rec, 1, S.desc[1]);
          pend |= 2u;
        }
      }
      __syncwarp();
      if (s_tk[0] < n_list) issue_J(S, J, pad, S.desc[0][0].z, S.desc[0][0].w, tid);
    }
    __syncthreads();
    if (s_tk[0] < n_list) {
      // t rows and V^-1 of the first tile
      const bool ok = mbar_wait(&S.mbR[0], parR & 1u, kCopyWaitCycles);
      if (ok) {
        parR ^= 1u;
        pend &= ~1u;
      } else {
        s_fail = 1;
      }
      const int4 d0 = S.desc[0][0], d1 = S.desc[0][1];
      const TileRecLayout g = tile_rec_layout(d0.w, d1.y, d0.y);
      const int* scam = reinterpret_cast<const int*>(&S.rec[0][g.scam]);
      if (ok && tid < d1.y) {  // the record's slot cameras are valid only once it has arrived
        const float* src = t_cam + (size_t)scam[tid] * kTStride;
        cp_async16(&S.tc[0][tid][0], src);
        cp_async16(&S.tc[0][tid][4], src + 4);
        cp_async16(&S.tc[0][tid][8], src + 8);
      }
      if (tid < d0.y) {
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_async4(&S.vi[0][tid][k], Vinv + (size_t)(d0.x + tid) * 6 + k);
      }
      cp_async_commit();
    }
    // ---- phase A, steady state: tile k uses desc[k % 4], rec[k % 3], tc / vi[k % 2]
    for (int k = 0;; ++k) {
      const int dk = k & 3, rk = k % 3, bk = k & 1;
      if (s_tk[dk] >= n_list || s_fail) break;
      if (mbar_wait(&S.mbJ, parJ, kCopyWaitCycles)) {
        parJ ^= 1u;
        pend &= ~8u;
      } else {
        s_fail = 1;
      }
      cp_async_wait_all();
      __syncthreads();
      if (s_fail) break;
      const int4 d0 = S.desc[dk][0], d1 = S.desc[dk][1];
      const int nl = d0.y, o0 = d0.z, n = d0.w, ns = d1.y;
      const TileRecLayout g = tile_rec_layout(n, ns, nl);
      const uint8_t* rec = S.rec[rk];
      const bool active = tid < n;
      float jp[18], jl[6];
      int meta = 0, lm = 0;
      if (active) {
        const int sh = (o0 & 3) + tid;
#pragma unroll
        for (int p = 0; p < 18; ++p) jp[p] = S.sJ[p][sh];
#pragma unroll
        for (int p = 0; p < 6; ++p) jl[p] = S.sJ[18 + p][sh];
        meta = reinterpret_cast<const uint16_t*>(rec + g.meta)[tid];
        lm = rec[g.olm + tid];
      }
      const int k1 = (k + 1) & 3, k2 = (k + 2) & 3, k3 = (k + 3) & 3;
      // after the core's first barrier every thread holds its J in registers and is past the
      // start of this tile: refill sJ, the record ring and the descriptor ring for the tiles
      // ahead, and fetch the next tile's t rows and V^-1 once its record has arrived
      auto ahead = [&]() {
        if (tid < 32) {
          if (s_tk[k1] < n_list) {
            issue_J(S, J, pad, S.desc[k1][0].z, S.desc[k1][0].w, tid);
            if (tid == 0) pend |= 8u;
          }
          if (tid == 0) {
            if (s_tk[k2] < n_list) {
              issue_rec(S, tp.tile_rec, (k + 2) % 3, S.desc[k2]);
              pend |= 1u << ((k + 2) % 3);
            }
            // the ticket claimed one tile ago (at or past n_list: none) and the all-stopped
            // flag read then: neither round trip is waited for in the tile that starts it
            const int tk = tk_next;
            s_tk[k3] = tk;
            tk_next = n_list;
            if (tk < n_list) {
              cp_async16(&S.desc[k3][0], list + 2 * (size_t)tk);
              cp_async16(&S.desc[k3][1], list + 2 * (size_t)tk + 1);
              if (!stop_seen) tk_next = (int)atomicAdd(&gs->tile_next, 1u);
            }
            stop_seen = ld_volatile(&sgl->all_done);
          }
        }
        if (s_tk[k1] >= n_list) {
          cp_async_commit();
          return;
        }
        const int r1 = (k + 1) % 3;
        const bool ok = mbar_wait(&S.mbR[r1], (parR >> r1) & 1u, kCopyWaitCycles);
        if (ok) {
          parR ^= 1u << r1;
          pend &= ~(1u << r1);
        } else {
          s_fail = 1;
        }
        const int4 e0 = S.desc[k1][0], e1 = S.desc[k1][1];
        const TileRecLayout h = tile_rec_layout(e0.w, e1.y, e0.y);
        const int* scam1 = reinterpret_cast<const int*>(&S.rec[r1][h.scam]);
        if (ok && tid < e1.y) {
          const float* src = t_cam + (size_t)scam1[tid] * kTStride;
          cp_async16(&S.tc[bk ^ 1][tid][0], src);
          cp_async16(&S.tc[bk ^ 1][tid][4], src + 4);
          cp_async16(&S.tc[bk ^ 1][tid][8], src + 8);
        }
        if (tid < e0.y) {
#pragma unroll
          for (int q = 0; q < 6; ++q)
            cp_async4(&S.vi[bk ^ 1][tid][q], Vinv + (size_t)(e0.x + tid) * 6 + q);
        }
        cp_async_commit();
      };
      f32_tile_core<kModeSeries, false>(active, n, ns, lm, meta, jp, jl, &S.tc[bk][0][0],
                                        kTStride, &S.vi[bk][0][0], 6,
                                        reinterpret_cast<const uint16_t*>(rec + g.sseg),
                                        reinterpret_cast<const uint16_t*>(rec + g.sbeg),
                                        reinterpret_cast<const int*>(rec + g.srow), S.sv, S.sg,
                                        partial, ahead);
    }
    cp_async_wait_all();
    __syncthreads();
    if (s_fail) {
      // let the bulk copies this block started finish (each wait bounded) before it leaves
      if (tid == 0) {
        atomicExch(&gs->error, 1);
        if (pend & 8u) mbar_wait(&S.mbJ, parJ, kCopyWaitCycles);
        for (int r = 0; r < 3; ++r)
          if (pend & (1u << r)) mbar_wait(&S.mbR[r], (parR >> r) & 1u, kCopyWaitCycles);
      }
      __syncthreads();
      return;
    }
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 1] = global_ns();
    if (!tile_end_barrier(gs, timeout, &s_last, &s_gen, &s_ok)) return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 2] = global_ns();
    if (tid == 0) s_done = ld_volatile(&sgl->all_done);
    __syncthreads();
    if (s_done) break;
    // ---- phase B: cameras
    camera_phase<float>(tp, cr, rc, partial, Uinv, x, t_cam, cam_norm, st, scratch);
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 3] = global_ns();
    if (!term_end_barrier(tp, gs, cam_norm, st, sgl, i, eps, timeout, &s_last, &s_gen, &s_ok,
                          &s_running))
      return;
    if (tracer && i <= kTraceTerms) trace[(i - 1) * kTracePoints + 4] = global_ns();
  }
  round_writeback(rc, x);
}

int persistent_blocks_per_sm(bool f32) {
  int nb = 0;
  if (f32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_kernel<float>, kTileObs, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_kernel<double>, kTileObs, 0);
  return nb;
}

int pipelined_blocks_per_sm() {
  if (cudaFuncSetAttribute(series_persistent_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(F32Pipe)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, series_persistent_f32_kernel, kTileObs,
                                                    sizeof(F32Pipe)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

template <typename T>
cudaError_t launch_series_persistent(const Topology& tp, const CamRounds& cr, int grid, const T* J, const T* Vinv,
                                     const double* Uinv, double* x, T* t_cam, T* partial,
                                     double* cam_norm, SeriesState* st, SeriesGlobal* sgl,
                                     GridSync* gs, int m_max, double eps, long long timeout,
                                     long long* trace, cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&cr, (void*)&J, (void*)&Vinv, (void*)&Uinv, (void*)&x,
                  (void*)&t_cam, (void*)&partial, (void*)&cam_norm, (void*)&st, (void*)&sgl,
                  (void*)&gs, (void*)&m_max, (void*)&eps, (void*)&timeout, (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_persistent_kernel<T>, dim3(grid),
                                     dim3(kTileObs), args, 0, s);
}

cudaError_t launch_series_pipelined(const Topology& tp, const CamRounds& cr, int grid,
                                    const int4* list,
                                    const int* n_list, const float* J, const float* Vinv,
                                    const double* Uinv, double* x, float* t_cam, float* partial,
                                    double* cam_norm, SeriesState* st, SeriesGlobal* sgl,
                                    GridSync* gs, int m_max, double eps, long long timeout,
                                    long long* trace, cudaStream_t s) {
  void* args[] = {(void*)&tp, (void*)&cr, (void*)&list, (void*)&n_list, (void*)&J, (void*)&Vinv,
                  (void*)&Uinv, (void*)&x, (void*)&t_cam, (void*)&partial, (void*)&cam_norm,
                  (void*)&st, (void*)&sgl, (void*)&gs, (void*)&m_max, (void*)&eps,
                  (void*)&timeout, (void*)&trace};
  return cudaLaunchCooperativeKernel((const void*)series_persistent_f32_kernel, dim3(grid),
                                     dim3(kTileObs), args, sizeof(F32Pipe), s);
}

template cudaError_t launch_series_persistent<double>(const Topology&, const CamRounds&, int, const double*, const double*, const double*, double*, double*, double*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);
template cudaError_t launch_series_persistent<float>(const Topology&, const CamRounds&, int, const float*, const float*, const double*, double*, float*, float*, double*, SeriesState*, SeriesGlobal*, GridSync*, int, double, long long, long long*, cudaStream_t);

}  // namespace poba
