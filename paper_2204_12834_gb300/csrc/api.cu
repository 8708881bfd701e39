// C ABI of libpoba (include/poba.h): handle life cycle, device arena, LM orchestration.
//
// One handle owns one problem on one GPU.  All device buffers live in a single arena
// allocated at creation; every call is ordered on the handle's stream.  The series loop
// (b~ and x(0), up to max_inner terms, back-substitution) is recorded once as a CUDA graph and
// replayed; terms after the stop rule fired return at kernel entry.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/poba.h"
#include "poba_internal.cuh"

using namespace poba;

namespace {

thread_local std::string g_last_error;

ba_status fail(ba_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ba_status fail_cuda(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error where possible
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA;
}

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail_cuda(e_, #call);           \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device address of one field of the device-resident LM record.
double* rec_field(LmRecord* rec, size_t offset) { return (double*)((char*)rec + offset); }

}  // namespace

void poba::set_last_error(const std::string& msg) { g_last_error = msg; }

struct ba_handle {
  int n_c = 0, n_l = 0, n_o = 0, n_o_pad = 0;
  int n_li = 0;  // internal landmarks: n_l plus the extra pieces of long tracks
  int precision = BA_FP64;
  bool weighted = false;
  ba_options opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Schedule sched;
  Topology tp{};

  void* arena = nullptr;
  size_t arena_bytes = 0;

  // problem (internal orders)
  double2* obs = nullptr;
  double* sqrt_w = nullptr;
  float2* obs32 = nullptr;     // FP32 bulk: float copies of obs and sqrt_w (linearisation)
  float* sqrt_w32 = nullptr;
  float* prep32 = nullptr;     // FP32 bulk: float copy of the prepared camera records
  double* cams = nullptr;
  double* cams_trial = nullptr;
  double* lms = nullptr;
  double* prep = nullptr;
  double* prep_trial = nullptr;
  // linearisation (bulk precision)
  void* J = nullptr;
  void* r = nullptr;
  void* partial = nullptr;
  void* t_cam = nullptr;  // current series term per camera-major slot row (bulk precision)
  double* U45 = nullptr;
  double* b_p = nullptr;
  double* V = nullptr;
  double* b_l = nullptr;
  // right-hand side the series solves with: (b_p, b_l) for a step of eq. `normal`, the adjoint
  // buffers (adj_p, adj_l) = -(dL/dx_p, dL/dx_l) for ba_adjoint
  const double* rhs_p = nullptr;
  const double* rhs_l = nullptr;
  double* adj_p = nullptr;
  double* adj_l = nullptr;
  int32_t* obs_caller = nullptr;   // [n_obs] caller index of each sorted observation
  int32_t* lm_order_dev = nullptr; // [n_lms] caller index of each internal landmark
  double* grad_out = nullptr;      // ba_adjoint host-output scratch [3 n_obs] (allocated on use)
  // PCG buffers (allocated on first use): y r z p q rhs [9 n_c], scalars, dot partials,
  // Schur-Jacobi blocks (sums, assembled, inverted)
  double* pcg = nullptr;
  double *pcg_y = nullptr, *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr, *pcg_q = nullptr,
         *pcg_rhs = nullptr, *pcg_sc = nullptr, *pcg_part = nullptr, *pcg_sj = nullptr,
         *pcg_s45 = nullptr, *pcg_minv = nullptr;
  double* Uinv = nullptr;
  double* Vinv = nullptr;
  float* Vinv_f = nullptr;
  // series
  double* x = nullptr;
  double* dx_l = nullptr;
  double* cam_norm = nullptr;     // (||t_c||^2, ||x_c||^2) per camera
  double* block_cost = nullptr;   // per tile: 2 F at the linearisation point
  double* tile_cost = nullptr;    // per tile: 2 F at a trial point
  double* block_pred = nullptr;   // per tile: 2 (L(0) - L(dx))
  double* scalars = nullptr;      // [0] lambda for explicit solves, [1] cost out
  double* prob_cost = nullptr;    // [n_probs] F per problem (ba_cost_batch)
  GridSync* gs = nullptr;         // persistent kernel: grid-barrier state
  long long* trace = nullptr;     // persistent kernel: phase timeline of its last block
  SeriesState* st = nullptr;      // [n_probs]
  SeriesGlobal* sgl = nullptr;
  LmRecord* rec = nullptr;        // [n_probs]
  int32_t* not_spd = nullptr;
  int32_t* io_bad = nullptr;      // [3] non-finite flags and the "state differs" flag of ba_set_params
  int32_t* relin = nullptr;       // 1: the next captured LM step linearises (set on the device)
  int n_probs = 1;
  std::vector<int32_t> cam_off_h, lm_off_h;  // caller numbering of the problems' cameras / landmarks

  // host staging (pinned)
  SeriesState* h_st = nullptr;   // [n_probs]
  SeriesGlobal* h_sgl = nullptr;
  GridSync* h_gs = nullptr;
  LmRecord* h_rec = nullptr;     // [n_probs]
  int32_t* h_flag = nullptr;
  int32_t* h_io = nullptr;       // [3]
  int32_t* h_relin = nullptr;    // host value written to relin before a captured step
  double* h_scalar = nullptr;

  bool linearized = false;
  // LM steps as one captured CUDA graph (linearisation gated on the device flag relin, the
  // solve, the evaluation and decision, the copies of the records to pinned host memory)
  bool step_graph = true;
  bool relin_synced = false;      // relin equals !linearized
  cudaGraphExec_t step_exec = nullptr;
  int step_kernels = 0;           // kernel nodes of the step graph
  int step_mode = 0;              // the series form captured in it
  std::vector<double> step_key;   // the configuration it was captured for
  bool cost_valid = false;
  bool have_step = false;
  bool last_solve_lm = false;  // the last solve was an LM step (per-problem lambdas)
  double solve_lambda = 0.0;   // lambda of the last explicit solve
  cudaGraphExec_t graph_exec = nullptr;
  int graph_max_inner = -1;
  double graph_eps = -1.0;
  int graph_nodes = 0;
  bool graph_timing = false;
  bool graph_active = false;
  const double* graph_rhs = nullptr;
  // series schedule (groups of chunks) and what depends on it, in a device allocation of its
  // own that is rebuilt when the group size changes: descriptors, records, group slots, the
  // series partial rows and the camera rounds of the persistent kernel for 1..plain_max blocks
  // per SM
  SerSchedule ser;
  SerTopo sp{};
  void* ser_arena = nullptr;
  size_t ser_bytes = 0;
  CheckRecord* chk = nullptr;  // debug-build check record (main arena)
  // debug builds: offsets of the guard bytes after each sub-buffer of the main (0) and series (1)
  // allocations, on the device
  uint64_t* canary_dev[2] = {nullptr, nullptr};
  int canary_n[2] = {0, 0};
  FlowState flow{};           // dataflow kernel state (inside ser_arena), zeroed per launch
  void* flow_base = nullptr;
  size_t flow_bytes = 0;
  void* ser_partial = nullptr;           // [n_gslots][9] partial rows (bulk precision)
  int group_obs = 0;                     // requested group size (0: automatic)
  int ser_long = 0;                      // series groups run by the long-group body
  // persistent kernel: grid = blocks per SM x SMs
  int sms = 0;
  int l2_bytes = 0;                      // L2 size of the device
  int plain_max = 0;                     // occupancy limit (0: kernel unavailable)
  int plain_k = 0;                       // blocks per SM in use
  int stage_max = 0, stage_k = 0;        // FP32 staged persistent kernel: limit, in use
  int flow_max = 0, flow_k = 0;          // dataflow persistent kernel: limit, in use
  CamRounds plain_rounds[4]{};           // per blocks-per-SM setting (1..4; any persistent form)
  int auto_exec = 1;                     // form used for series_exec 2: 1, 3, 4 or 5
  long long barrier_timeout = 1LL << 33;  // clock cycles a block waits at a grid barrier
  int last_exec = -1;                    // execution form of the last solve (1, 0, 3 or 4)
  uint64_t launches = 0;

  // kernel timing: event pairs per class; series classes have one pair per term
  bool timing = false;
  bool capturing = false;
  bool capturing_step = false;    // capturing an LM step (the series runs as per-term launches)
  int timing_terms = -1;
  std::vector<cudaEvent_t> ev;  // layout: see ev_index()
  double t_ms[BA_TIMING_CLASSES] = {0};
  uint64_t t_count[BA_TIMING_CLASSES] = {0};
  bool pending[BA_TIMING_CLASSES] = {false};

  bool f32() const { return precision == BA_FP32_BULK; }
};

namespace poba {
// *differ |= 1 if the input state differs from the current one in any bit (kernels_series.cu;
// order: the internal landmark rows' caller rows, 3 values each; null for cameras).
void launch_state_differs(const double* src, const double* cur, const int32_t* order, int n,
                          int32_t* differ, cudaStream_t s);
}  // namespace poba

namespace {

bool valid_options(const ba_options& o, std::string* why) {
  if (!(o.lambda0 > 0.0) || !std::isfinite(o.lambda0)) { *why = "lambda0 must be > 0"; return false; }
  if (!(o.func_tol >= 0.0)) { *why = "func_tol must be >= 0"; return false; }
  if (!(o.eps >= 0.0)) { *why = "eps must be >= 0"; return false; }
  if (o.max_lm < 0 || o.max_lm > 100000) { *why = "max_lm out of range"; return false; }
  if (o.max_inner < 0 || o.max_inner > 10000) { *why = "max_inner out of range [0, 10000]"; return false; }
  if (o.damping_mode != 0 && o.damping_mode != 1) { *why = "damping_mode must be 0 or 1"; return false; }
  if (o.series_exec < 0 || o.series_exec > 5) { *why = "series_exec must be in [0, 5]"; return false; }
  return true;
}

template <typename T>
void copy_in(std::vector<T>& dst, const T* src, size_t n, int ptr_kind) {
  dst.resize(n);
  if (n == 0) return;
  if (ptr_kind == 1) cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost);
  else std::memcpy(dst.data(), src, n * sizeof(T));
}

// Write a host vector to a caller pointer of the given kind.
ba_status copy_out(void* dst, const void* src, size_t bytes, int ptr_kind) {
  if (bytes == 0) return BA_OK;
  if (ptr_kind == 1) CK(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
  else std::memcpy(dst, src, bytes);
  return BA_OK;
}

ba_status debug_verify(ba_handle* h);

// NVTX range over a scope (host side: the calls that launch a kernel class, and each LM
// iteration), for profilers that filter by range; free when no tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

ba_status check_launch(ba_handle* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_cuda(e, what);
  return debug_verify(h);
}

// Debug builds (checks.cuh): guard bytes after each sub-buffer of an allocation.  layout:
// returns the bytes a sub-buffer of `bytes` takes (its guard included); fill: writes the guard
// bytes at the given offsets and uploads the offsets for the check kernel.
size_t guarded(size_t bytes) { return bytes + (kChecks ? kCanaryBytes : 0); }

cudaError_t install_canaries(ba_handle* h, int which, void* base,
                             const std::vector<uint64_t>& offs) {
  if (!kChecks) return cudaSuccess;
  for (uint64_t o : offs) {
    cudaError_t e = cudaMemset((char*)base + o, kCanaryByte, kCanaryBytes);
    if (e != cudaSuccess) return e;
  }
  if (h->canary_dev[which]) cudaFree(h->canary_dev[which]);
  h->canary_dev[which] = nullptr;
  h->canary_n[which] = (int)offs.size();
  if (offs.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(&h->canary_dev[which], sizeof(uint64_t) * offs.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(h->canary_dev[which], offs.data(), sizeof(uint64_t) * offs.size(),
                   cudaMemcpyHostToDevice);
  return e;
}

// Debug builds: after the handle's stream drains, the guard bytes of both allocations and the
// device check record; the first failure becomes BA_ERR_CHECK (the record is then cleared, so
// the handle stays usable).  Release builds, and while a graph is being captured: BA_OK.
ba_status debug_verify(ba_handle* h) {
  if (!kChecks || h->capturing || !h->chk) return BA_OK;
  cudaStream_t s = h->stream;
  if (h->canary_n[0] > 0)
    launch_canary_check((const uint8_t*)h->arena, h->canary_dev[0], h->canary_n[0], kChkCanary,
                        h->chk, s);
  if (h->canary_n[1] > 0 && h->ser_arena)
    launch_canary_check((const uint8_t*)h->ser_arena, h->canary_dev[1], h->canary_n[1],
                        kChkCanary + 1000, h->chk, s);
  CheckRecord r{};
  cudaError_t e = cudaMemcpyAsync(&r, h->chk, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda(e, "device check record");
  if (r.site == kChkNone) return BA_OK;
  cudaMemsetAsync(h->chk, 0, sizeof(CheckRecord), s);
  return fail(BA_ERR_CHECK, "device check " + std::to_string(r.site) + " failed: index " +
                                std::to_string(r.index) + " for bound " + std::to_string(r.bound) +
                                " (" + std::to_string(r.count) + " failed checks)");
}

// ---- kernel timing --------------------------------------------------------------------
// Event pair index: classes 0, 1, 2, 5, 6 own one pair; classes 3 and 4 own one pair per term.
enum { kTLin = 0, kTDamp = 1, kTRhs = 2, kTTile = 3, kTCam = 4, kTBack = 5, kTEval = 6 };

int ev_index(const ba_handle* h, int cls, int term) {
  const int M = h->timing_terms;
  switch (cls) {
    case kTLin: return 0;
    case kTDamp: return 2;
    case kTRhs: return 4;
    case kTBack: return 6;
    case kTEval: return 8;
    case kTTile: return 10 + 2 * (term - 1);
    default: return 10 + 2 * M + 2 * (term - 1);
  }
}

ba_status ensure_events(ba_handle* h) {
  if (h->timing_terms == h->opts.max_inner && !h->ev.empty()) return BA_OK;
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
  h->timing_terms = h->opts.max_inner;
  const int n = 10 + 4 * h->opts.max_inner;
  h->ev.resize(n);
  for (int i = 0; i < n; ++i) CK(cudaEventCreate(&h->ev[i]));
  return BA_OK;
}

// Record the start (which = 0) or end (1) event of a timed class on the handle's stream.
void tmark(ba_handle* h, int cls, int term, int which) {
  if (!h->timing) return;
  cudaEvent_t e = h->ev[ev_index(h, cls, term) + which];
  if (h->capturing) cudaEventRecordWithFlags(e, h->stream, cudaEventRecordExternal);
  else cudaEventRecord(e, h->stream);
  if (which == 1 && cls != kTTile && cls != kTCam) h->pending[cls] = true;
}

// After a stream synchronisation: add the elapsed time of every pair that ran.
void collect_timing(ba_handle* h, int terms_run, bool series_ran) {
  if (!h->timing) return;
  float ms = 0.f;
  for (int cls : {kTLin, kTDamp, kTRhs, kTBack, kTEval}) {
    if (!h->pending[cls]) continue;
    const int i = ev_index(h, cls, 0);
    if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) {
      h->t_ms[cls] += ms;
      h->t_count[cls] += 1;
    }
    h->pending[cls] = false;
  }
  if (series_ran && h->last_exec >= 3) {
    // one pair around the persistent kernel, counted once per executed term
    const int i = ev_index(h, kTTile, 1);
    if (terms_run >= 1 && cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) {
      h->t_ms[kTTile] += ms;
      h->t_count[kTTile] += (uint64_t)terms_run;
    }
  } else if (series_ran) {
    for (int term = 1; term <= terms_run && term <= h->timing_terms; ++term) {
      for (int cls : {kTTile, kTCam}) {
        const int i = ev_index(h, cls, term);
        if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) {
          h->t_ms[cls] += ms;
          h->t_count[cls] += 1;
        }
      }
    }
  }
  cudaGetLastError();
}

// ---- kernel sequences ------------------------------------------------------------------

// Extra kernel of a step for the long tracks of a handle (their block and back-substitution
// kernels), 0 without long tracks.
int long_kernels(const ba_handle* h) { return h->tp.n_long > 0 ? 1 : 0; }
// The staged and dataflow series kernels take groups of whole landmarks within the slot cap only:
// none of long tracks' pieces or of landmarks wider than the cap.
bool has_long_groups(const ba_handle* h) { return h->tp.n_long > 0 || h->ser_long > 0; }

void seq_linearize(ba_handle* h) {
  Range range("poba.linearize");
  cudaStream_t s = h->stream;
  tmark(h, kTLin, 0, 0);
  launch_cam_prepare(h->cams, nullptr, h->n_c, h->prep, nullptr, s, h->prep32);
  if (h->f32()) {
    launch_linearize<float>(h->tp, h->prep32, h->lms, h->obs32, h->sqrt_w32, (float*)h->J,
                            (float*)h->r, h->V, h->b_l, (float*)h->partial, h->block_cost, s);
    launch_lin_camera_reduce<float>(h->tp, (const float*)h->partial, h->U45, h->b_p, s);
  } else {
    launch_linearize<double>(h->tp, h->prep, h->lms, h->obs, h->sqrt_w, (double*)h->J,
                             (double*)h->r, h->V, h->b_l, (double*)h->partial, h->block_cost, s);
    launch_lin_camera_reduce<double>(h->tp, (const double*)h->partial, h->U45, h->b_p, s);
  }
  launch_long_track_blocks(h->tp, h->V, h->b_l, s);
  tmark(h, kTLin, 0, 1);
  h->launches += 3 + long_kernels(h);
}

// series reset, b~ / x(0), max_inner terms, back-substitution with model decrease
template <typename T>
void seq_series_body(ba_handle* h, cudaStream_t s, bool use_active) {
  const Topology& tp = h->tp;
  const SerTopo& sp = h->sp;
  const T* J = (const T*)h->J;
  const T* Vi = h->f32() ? (const T*)(const void*)h->Vinv_f : (const T*)(const void*)h->Vinv;
  T* part = (T*)h->ser_partial;
  launch_series_reset(h->st, h->sgl, use_active ? h->rec : nullptr, h->n_probs, s);
  tmark(h, kTRhs, 0, 0);
  launch_tile_rhs<T>(tp, sp, J, h->rhs_l, Vi, part, h->st, s);
  launch_camera_rhs<T>(tp, sp, part, h->rhs_p, h->Uinv, h->x, (T*)h->t_cam, h->cam_norm, h->st,
                       h->sgl, s);
  tmark(h, kTRhs, 0, 1);
  for (int i = 1; i <= h->opts.max_inner; ++i) {
    tmark(h, kTTile, i, 0);
    launch_tile_series<T>(tp, sp, J, (const T*)h->t_cam, Vi, part, h->st, h->sgl, s);
    tmark(h, kTTile, i, 1);
    tmark(h, kTCam, i, 0);
    launch_camera_series<T>(tp, sp, part, h->Uinv, h->x, (T*)h->t_cam, h->cam_norm, h->st,
                            h->sgl, i, h->opts.eps, s);
    tmark(h, kTCam, i, 1);
  }
  tmark(h, kTBack, 0, 0);
  launch_tile_backsub<T>(tp, J, (const T*)h->r, h->x, h->rhs_l, Vi, h->dx_l, h->block_pred, s);
  tmark(h, kTBack, 0, 1);
}

// Kernels of one series solve in the per-term forms (the group kernel is skipped when the
// schedule has no group).
int series_body_kernels(const ba_handle* h) {
  const int group = h->sp.n_groups > 0 ? 1 : 0;
  return 3 + group + long_kernels(h) + (1 + group) * h->opts.max_inner;
}

template <typename T>
ba_status seq_series_persistent(ba_handle* h, cudaStream_t s, bool use_active, int form) {
  const bool staged = form == 4, flow = form == 5;
  const Topology& tp = h->tp;
  const SerTopo& sp = h->sp;
  const T* J = (const T*)h->J;
  const T* Vi = h->f32() ? (const T*)(const void*)h->Vinv_f : (const T*)(const void*)h->Vinv;
  T* part = (T*)h->ser_partial;
  launch_series_reset(h->st, h->sgl, use_active ? h->rec : nullptr, h->n_probs, s);
  tmark(h, kTRhs, 0, 0);
  launch_tile_rhs<T>(tp, sp, J, h->rhs_l, Vi, part, h->st, s);
  launch_camera_rhs<T>(tp, sp, part, h->rhs_p, h->Uinv, h->x, (T*)h->t_cam, h->cam_norm, h->st,
                       h->sgl, s);
  tmark(h, kTRhs, 0, 1);
  // reset, the RHS kernels, back-substitution (and that of the long tracks)
  h->launches += 3 + (sp.n_groups > 0 ? 1 : 0) + long_kernels(h);
  CK(cudaMemsetAsync(h->gs, 0, sizeof(GridSync), s));
  if (flow) {
    CK(cudaMemsetAsync(h->flow_base, 0, h->flow_bytes, s));
    CK(cudaMemsetAsync(h->trace, 0, sizeof(long long) * kTraceTerms * kTracePoints, s));
  }
  if (h->opts.max_inner > 0) {
    tmark(h, kTTile, 1, 0);
    if constexpr (sizeof(T) == 4) {
      if (staged) {
        CK(launch_series_staged(tp, sp, h->plain_rounds[h->stage_k - 1], h->stage_k * h->sms, J,
                                Vi, h->Uinv, h->x, (T*)h->t_cam, part, h->cam_norm, h->st,
                                h->sgl, h->gs, h->opts.max_inner, h->opts.eps,
                                h->barrier_timeout, h->trace, s));
      }
    }
    if (flow) {
      CK(launch_series_dataflow<T>(tp, sp, h->flow, h->flow_k * h->sms, J, Vi, h->Uinv, h->x,
                                   (T*)h->t_cam, part, h->cam_norm, h->st, h->sgl, h->gs,
                                   h->opts.max_inner, h->opts.eps, h->barrier_timeout, h->trace,
                                   s));
    } else if (!staged) {
      CK(launch_series_persistent<T>(tp, sp, h->plain_rounds[h->plain_k - 1],
                                     h->plain_k * h->sms, J, Vi, h->Uinv, h->x, (T*)h->t_cam,
                                     part, h->cam_norm, h->st, h->sgl, h->gs, h->opts.max_inner,
                                     h->opts.eps, h->barrier_timeout, h->trace, s));
    }
    tmark(h, kTTile, 1, 1);
    h->launches += 1;
  }
  tmark(h, kTBack, 0, 0);
  launch_tile_backsub<T>(tp, J, (const T*)h->r, h->x, h->rhs_l, Vi, h->dx_l, h->block_pred, s);
  tmark(h, kTBack, 0, 1);
  return BA_OK;
}

ba_status run_series_body(ba_handle* h, bool use_active) {
  Range range("poba.series");
  cudaStream_t s = h->stream;
  if (h->timing) {
    ba_status st = ensure_events(h);
    if (st != BA_OK) return st;
  }
  // execution form: 0 per-term launches, 1 graph replay, 3 persistent, 4 persistent with staged
  // chunks (FP32 bulk); series_exec 2 takes the handle's schedule (default or ba_autotune)
  int mode = h->opts.series_exec == 2 ? h->auto_exec : h->opts.series_exec;
  // the dataflow kernel numbers its tickets (term, group) in 32 bits
  // (the staged and dataflow kernels take no long groups: has_long_groups)
  if (mode == 5 && (h->flow_k <= 0 || has_long_groups(h) ||
                    (int64_t)h->opts.max_inner * h->sp.n_groups >= (1LL << 31)))
    mode = 3;
  if (mode == 4 && (h->stage_k <= 0 || has_long_groups(h))) mode = 3;
  if (mode == 3 && h->plain_k <= 0) mode = 1;
  if (mode == 1 && h->capturing_step) mode = 0;  // the step graph holds the per-term launches
  h->last_exec = mode;
  if (mode >= 3) {
    ba_status st = h->f32() ? seq_series_persistent<float>(h, s, use_active, mode)
                            : seq_series_persistent<double>(h, s, use_active, mode == 4 ? 3 : mode);
    if (st == BA_OK) h->pending[kTRhs] = h->pending[kTBack] = h->timing;
    return st;
  }
  if (mode == 1) {
    if (!h->graph_exec || h->graph_max_inner != h->opts.max_inner || h->graph_eps != h->opts.eps ||
        h->graph_timing != h->timing || h->graph_active != use_active ||
        h->graph_rhs != h->rhs_p) {
      if (h->graph_exec) {
        cudaGraphExecDestroy(h->graph_exec);
        h->graph_exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      h->capturing = true;
      if (h->f32()) seq_series_body<float>(h, s, use_active);
      else seq_series_body<double>(h, s, use_active);
      h->capturing = false;
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&h->graph_exec, g, 0);
      size_t nn = 0;
      cudaGraphGetNodes(g, nullptr, &nn);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return fail_cuda(e, "cudaGraphInstantiate");
      h->graph_nodes = (int)nn;
      h->graph_max_inner = h->opts.max_inner;
      h->graph_eps = h->opts.eps;
      h->graph_timing = h->timing;
      h->graph_active = use_active;
      h->graph_rhs = h->rhs_p;
    }
    CK(cudaGraphLaunch(h->graph_exec, s));
    if (h->timing) {
      h->pending[kTRhs] = true;
      h->pending[kTBack] = true;
    }
    h->launches += (uint64_t)series_body_kernels(h);
  } else {
    if (h->f32()) seq_series_body<float>(h, s, use_active);
    else seq_series_body<double>(h, s, use_active);
    h->launches += (uint64_t)series_body_kernels(h);
  }
  return BA_OK;
}

// lambda of problem p at lam_dev[p * lam_stride]; use_active: problems whose LM record is
// inactive take no part.
ba_status run_solve(ba_handle* h, const double* lam_dev, int lam_stride, bool use_active) {
  Range range("poba.solve");
  CK(cudaMemsetAsync(h->not_spd, 0, sizeof(int32_t) * h->n_probs, h->stream));
  if (h->timing) {
    ba_status st = ensure_events(h);
    if (st != BA_OK) return st;
  }
  tmark(h, kTDamp, 0, 0);
  launch_damp_invert(h->tp, h->U45, h->V, lam_dev, lam_stride, h->opts.damping_mode, h->Uinv,
                     h->Vinv, h->f32() ? h->Vinv_f : nullptr, h->not_spd, h->stream);
  tmark(h, kTDamp, 0, 1);
  h->launches += 1;
  ba_status st = run_series_body(h, use_active);
  if (st != BA_OK) return st;
  h->have_step = true;
  return check_launch(h, "series kernels");
}

// F(x) per problem at the current state into out[p * stride] (fixed order).
void seq_cost(ba_handle* h, double* out, int stride) {
  launch_cam_prepare(h->cams, nullptr, h->n_c, h->prep, nullptr, h->stream);
  launch_tile_cost(h->tp, h->prep, h->lms, nullptr, h->obs, h->sqrt_w, h->tile_cost, h->stream);
  launch_reduce_tiles(h->tp, h->tile_cost, out, stride, 0.5, h->stream);
  h->launches += 3;
}

constexpr int kRecStride = (int)(sizeof(LmRecord) / sizeof(double));

}  // namespace

extern "C" {

ba_status ba_default_options(ba_options* o) {
  if (!o) return fail(BA_ERR_INVALID_ARG, "opts is NULL");
  o->lambda0 = 1e-4;
  o->func_tol = 1e-6;
  o->eps = 0.01;
  o->max_lm = 50;
  o->max_inner = 20;
  o->damping_mode = 0;
  o->series_exec = 2;
  return BA_OK;
}

ba_status ba_destroy(ba_handle* h) {
  if (!h) return BA_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->arena) cudaFree(h->arena);
  if (h->ser_arena) cudaFree(h->ser_arena);
  for (uint64_t* c : h->canary_dev)
    if (c) cudaFree(c);
  if (h->grad_out) cudaFree(h->grad_out);
  if (h->pcg) cudaFree(h->pcg);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_sgl) cudaFreeHost(h->h_sgl);
  if (h->h_rec) cudaFreeHost(h->h_rec);
  if (h->h_gs) cudaFreeHost(h->h_gs);
  if (h->h_flag) cudaFreeHost(h->h_flag);
  if (h->h_io) cudaFreeHost(h->h_io);
  if (h->h_relin) cudaFreeHost(h->h_relin);
  if (h->h_scalar) cudaFreeHost(h->h_scalar);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return BA_OK;
}

}  // extern "C"

namespace {

// The blocks that run groups in the persistent kernel at its largest residency (the grid's last
// block applies the stop rule and takes no groups): the automatic group size is cut for them.
// Groups the automatic group size aims at for `blocks` blocks that run groups: one per block for
// a single problem; two per block for a batch, whose groups cannot span problems and whose
// problems stop at different terms and LM steps (with one group per block the blocks that hold
// stopped problems' groups idle; measured on the 256-problem batch: 705 against 603 problems/s).
int auto_groups(const ba_handle* h, int blocks) { return h->n_probs > 1 ? 2 * blocks : blocks; }
int auto_workers(const ba_handle* h) {
  return auto_groups(h, (h->plain_max > 0 ? h->plain_max : 2) * h->sms - 1);
}

// Default tail split of the series groups: none (ba_autotune tries splits).
constexpr int kDefaultTail = 0;

// (Re)builds the series schedule for a group size (0: automatic, n_obs / grid) and its device
// allocation: descriptors, chunk records, group slots, partial rows, and the camera rounds of
// the persistent kernel for each residency.  The old allocation is freed after the handle's
// stream drains, and the captured graph (which holds its pointers) is dropped.
ba_status rebuild_series(ba_handle* h, int group_obs, int tail) {
  const Schedule& S = h->sched;
  const int target = group_obs > 0 ? group_obs : series_auto_target(h->n_o, auto_workers(h));
  SerSchedule Q;
  const std::string why =
      build_series_schedule(S, target, tail, &Q, h->f32() ? kGroupSlots : kGroupSlotsF64);
  if (!why.empty()) return fail(BA_ERR_INVALID_ARG, why);
  CamSchedule cs;
  build_cam_schedule(Q.cam_ptr, h->n_c, &cs);
  CamRoundList rl[4];
  for (int k = 1; k <= h->plain_max && k <= 4; ++k) build_cam_rounds(cs, h->n_c, k * h->sms, &rl[k - 1]);
  const size_t bulk = h->f32() ? sizeof(float) : sizeof(double);
  struct Item { void** ptr; const void* src; size_t bytes; };
  int32_t *d_group = nullptr, *d_chunk = nullptr, *d_gcam = nullptr, *d_grow = nullptr,
          *d_cptr = nullptr, *d_item = nullptr, *d_q = nullptr, *d_rl[4][3] = {},
          *d_pnc = nullptr;
  uint8_t* d_rec = nullptr;
  void* d_part = nullptr;
  void* d_flow = nullptr;
  const size_t flow_bytes = flow_state_bytes(h->n_c, h->n_probs);
  auto nz = [](size_t b) { return b > 0 ? b : (size_t)16; };
  std::vector<Item> items = {
      {(void**)&d_group, Q.group.data(), sizeof(int32_t) * Q.group.size()},
      {(void**)&d_chunk, Q.chunk.data(), sizeof(int32_t) * Q.chunk.size()},
      {(void**)&d_rec, Q.rec.data(), Q.rec.size()},
      {(void**)&d_gcam, Q.gslot_cam.data(), sizeof(int32_t) * Q.gslot_cam.size()},
      {(void**)&d_grow, Q.gslot_row.data(), sizeof(int32_t) * Q.gslot_row.size()},
      {(void**)&d_cptr, Q.cam_ptr.data(), sizeof(int32_t) * Q.cam_ptr.size()},
      {(void**)&d_pnc, Q.prob_ncam.data(), sizeof(int32_t) * Q.prob_ncam.size()},
      {&d_part, nullptr, bulk * 9 * (size_t)Q.n_gslots},
      {&d_flow, nullptr, flow_bytes},
      {(void**)&d_item, cs.cam_item.data(), sizeof(int32_t) * cs.cam_item.size()},
      {(void**)&d_q, cs.item_q.data(), sizeof(int32_t) * cs.item_q.size()},
  };
  for (int k = 0; k < 4; ++k) {
    if (rl[k].round_cam.empty()) continue;
    items.push_back({(void**)&d_rl[k][0], rl[k].round_cam.data(), sizeof(int32_t) * rl[k].round_cam.size()});
    items.push_back({(void**)&d_rl[k][1], rl[k].round_item.data(), sizeof(int32_t) * rl[k].round_item.size()});
    items.push_back({(void**)&d_rl[k][2], rl[k].block_round.data(), sizeof(int32_t) * rl[k].block_round.size()});
  }
  size_t total = 0;
  for (auto& it : items) total = align_up(total, 256) + guarded(nz(it.bytes));
  total = align_up(total, 256);
  void* arena = nullptr;
  cudaError_t e = cudaMalloc(&arena, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(BA_ERR_OOM, "cudaMalloc(series schedule) failed");
  }
  size_t off = 0;
  std::vector<uint64_t> guards;
  for (auto& it : items) {
    off = align_up(off, 256);
    *it.ptr = (char*)arena + off;
    off += nz(it.bytes);
    if (kChecks) {
      guards.push_back(off);
      off += kCanaryBytes;
    }
  }
  // the old schedule may still be in use by queued work of the handle's stream
  e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemset(arena, 0, total);
  for (auto& it : items)
    if (e == cudaSuccess && it.src && it.bytes) e = cudaMemcpy(*it.ptr, it.src, it.bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = install_canaries(h, 1, arena, guards);
  if (e != cudaSuccess) {
    cudaFree(arena);
    return fail_cuda(e, "uploading the series schedule");
  }
  if (h->ser_arena) cudaFree(h->ser_arena);
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  if (h->step_exec) {
    cudaGraphExecDestroy(h->step_exec);
    h->step_exec = nullptr;
  }
  h->ser_arena = arena;
  h->ser_bytes = total;
  h->ser_partial = d_part;
  h->group_obs = group_obs;
  h->ser_long = Q.n_long_groups;
  // group bodies prefetch their next chunk when the Jacobians take more than half of L2 (each
  // term then streams much of them from HBM); an L2-resident problem gains nothing from it
  const size_t j_bytes = (size_t)24 * h->n_o_pad * (h->f32() ? 4 : 8);
  h->sp = SerTopo{Q.n_groups, Q.n_chunks, Q.n_gslots, (const int4*)d_group, (const int4*)d_chunk,
                  d_rec, d_gcam, d_grow, d_cptr, d_pnc, 2 * j_bytes > (size_t)h->l2_bytes ? 1 : 0};
  {
    // flow state: cam_norm_b first (16-byte pairs), then the counters
    char* f = (char*)d_flow;
    h->flow.cam_norm_b = (double*)f;
    f += (size_t)h->n_c * 16;
    h->flow.cam_cnt = (unsigned*)f;
    f += (size_t)h->n_c * 4;
    h->flow.cam_epoch = (int*)f;
    f += (size_t)h->n_c * 4;
    h->flow.pcnt = (unsigned*)f;
    f += (size_t)h->n_probs * 8;
    h->flow.prob_dec = (int*)f;
    h->flow_base = d_flow;
    h->flow_bytes = flow_bytes;
  }
  for (int k = 0; k < 4; ++k) h->plain_rounds[k] = CamRounds{d_item, d_q, d_rl[k][0], d_rl[k][1], d_rl[k][2]};
  h->ser = std::move(Q);
  return BA_OK;
}

// ba_create and ba_create_batch: the problems are concatenated (cameras, landmarks and
// observations of problem p follow those of problem p - 1, with indices offset to match) and
// scheduled so that no tile holds two problems.
ba_status create_impl(const ba_problem_desc* descs, int n_probs, const ba_options* opts,
                      ba_handle** out) {
  if (!out) return fail(BA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!descs) return fail(BA_ERR_INVALID_ARG, "desc is NULL");
  if (n_probs < 1) return fail(BA_ERR_INVALID_ARG, "n_problems must be >= 1");
  const int precision = descs[0].precision;
  int64_t tc = 0, tl = 0, to = 0;
  bool weighted = false;
  for (int p = 0; p < n_probs; ++p) {
    const ba_problem_desc* d = &descs[p];
    const std::string pre = n_probs > 1 ? "problem " + std::to_string(p) + ": " : "";
    if (d->n_cams < 1 || d->n_lms < 1 || d->n_obs < 0)
      return fail(BA_ERR_INVALID_ARG, pre + "need n_cams >= 1, n_lms >= 1, n_obs >= 0");
    if (d->ptr_kind != 0 && d->ptr_kind != 1)
      return fail(BA_ERR_INVALID_ARG, pre + "ptr_kind must be 0 or 1");
    if (d->precision != BA_FP64 && d->precision != BA_FP32_BULK)
      return fail(BA_ERR_INVALID_ARG, pre + "precision must be BA_FP64 or BA_FP32_BULK");
    if (d->precision != precision)
      return fail(BA_ERR_INVALID_ARG, pre + "all problems of a batch need the same precision");
    if (!d->cams || !d->lms) return fail(BA_ERR_INVALID_ARG, pre + "cams / lms is NULL");
    if (d->n_obs > 0 && (!d->obs || !d->cam_idx || !d->lm_idx))
      return fail(BA_ERR_INVALID_ARG, pre + "obs / cam_idx / lm_idx is NULL");
    tc += d->n_cams;
    tl += d->n_lms;
    to += d->n_obs;
    weighted = weighted || d->weights != nullptr;
  }
  if (tc > (1 << 28) || tl > (1 << 28) || to > (1LL << 31) - 128)
    return fail(BA_ERR_INVALID_ARG, "problem too large (cameras, landmarks < 2^28, observations < 2^31)");
  ba_options o;
  ba_default_options(&o);
  if (opts) o = *opts;
  std::string why;
  if (!valid_options(o, &why)) return fail(BA_ERR_INVALID_ARG, why);

  const int nc = (int)tc, nl = (int)tl, no = (int)to;
  std::vector<double> cams, lms, obs, w;
  std::vector<int32_t> ci, li, cam_off(n_probs + 1, 0), lm_off(n_probs + 1, 0);
  cams.reserve((size_t)nc * 9);
  lms.reserve((size_t)nl * 3);
  obs.reserve((size_t)no * 2);
  ci.reserve(no);
  li.reserve(no);
  if (weighted) w.reserve(no);
  for (int p = 0; p < n_probs; ++p) {
    const ba_problem_desc* d = &descs[p];
    const std::string pre = n_probs > 1 ? "problem " + std::to_string(p) + ": " : "";
    std::vector<double> c1, l1, o1, w1;
    std::vector<int32_t> ci1, li1;
    copy_in(c1, d->cams, (size_t)d->n_cams * 9, d->ptr_kind);
    copy_in(l1, d->lms, (size_t)d->n_lms * 3, d->ptr_kind);
    copy_in(o1, d->obs, (size_t)d->n_obs * 2, d->ptr_kind);
    copy_in(ci1, d->cam_idx, (size_t)d->n_obs, d->ptr_kind);
    copy_in(li1, d->lm_idx, (size_t)d->n_obs, d->ptr_kind);
    if (d->weights) copy_in(w1, d->weights, (size_t)d->n_obs, d->ptr_kind);
    if (d->ptr_kind == 1) {
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return fail_cuda(e, "copying device inputs");
    }
    for (double v : c1) if (!std::isfinite(v)) return fail(BA_ERR_NONFINITE, pre + "non-finite camera parameter");
    for (double v : l1) if (!std::isfinite(v)) return fail(BA_ERR_NONFINITE, pre + "non-finite landmark");
    for (double v : o1) if (!std::isfinite(v)) return fail(BA_ERR_NONFINITE, pre + "non-finite observation");
    for (double v : w1)
      if (!(v > 0.0) || !std::isfinite(v)) return fail(BA_ERR_INVALID_ARG, pre + "weights must be finite and > 0");
    if (n_probs > 1) {
      // index ranges are checked per problem before the offsets are added
      for (int k = 0; k < d->n_obs; ++k) {
        if (ci1[k] < 0 || ci1[k] >= d->n_cams)
          return fail(BA_ERR_INVALID_ARG, pre + "cam_idx[" + std::to_string(k) + "] out of range");
        if (li1[k] < 0 || li1[k] >= d->n_lms)
          return fail(BA_ERR_INVALID_ARG, pre + "lm_idx[" + std::to_string(k) + "] out of range");
      }
    }
    const int32_t c0 = cam_off[p], l0 = lm_off[p];
    cams.insert(cams.end(), c1.begin(), c1.end());
    lms.insert(lms.end(), l1.begin(), l1.end());
    obs.insert(obs.end(), o1.begin(), o1.end());
    for (int k = 0; k < d->n_obs; ++k) {
      ci.push_back(ci1[k] + c0);
      li.push_back(li1[k] + l0);
    }
    if (weighted) {
      if (d->weights) w.insert(w.end(), w1.begin(), w1.end());
      else w.insert(w.end(), (size_t)d->n_obs, 1.0);
    }
    cam_off[p + 1] = c0 + d->n_cams;
    lm_off[p + 1] = l0 + d->n_lms;
  }

  ba_handle* h = new ba_handle();
  h->n_c = nc;
  h->n_l = nl;
  h->n_o = no;
  h->n_o_pad = (int)align_up((size_t)(no > 0 ? no : 1), 64);
  h->precision = precision;
  h->weighted = weighted;
  h->opts = o;
  h->n_probs = n_probs;
  h->cam_off_h = cam_off;
  h->lm_off_h = lm_off;
  why = build_schedule(nc, nl, no, ci.data(), li.data(), n_probs, cam_off.data(), lm_off.data(),
                       &h->sched);
  if (!why.empty()) {
    delete h;
    return fail(BA_ERR_INVALID_ARG, why);
  }
  const Schedule& S = h->sched;
  const int nli = S.n_lms_int;  // internal landmark arrays (a long track has several pieces)
  h->n_li = nli;
  std::vector<int32_t> tile_prob(S.n_tiles);
  for (int t = 0; t < S.n_tiles; ++t) tile_prob[t] = S.lm_prob[S.tile_lm0[t]];

  {
    // persistent series kernel: all blocks must be co-resident (cooperative launch)
    int dev = 0, sms = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, dev);
    const int per_sm = persistent_blocks_per_sm(h->f32());
    h->sms = sms;
    // FP32 bulk: up to 4 blocks of 256 threads per SM, FP64: up to 3
    const int cap = h->f32() ? 4 : 3;
    h->plain_max = (coop && per_sm > 0) ? (per_sm < cap ? per_sm : cap) : 0;
    h->plain_k = h->plain_max;
    if (h->f32() && h->plain_max > 0) {
      const int st = staged_blocks_per_sm();
      h->stage_max = st < 3 ? st : 3;
      h->stage_k = h->stage_max;
    }
    if (coop) {
      const int fl = h->f32() ? dataflow_blocks_per_sm<float>() : dataflow_blocks_per_sm<double>();
      h->flow_max = fl > 0 ? (fl < cap ? fl : cap) : 0;
      h->flow_k = h->flow_max;
    }
    // default form: the persistent kernel at its largest residency; ba_autotune measures the
    // forms instead
    h->auto_exec = h->plain_k > 0 ? 3 : 1;
    cudaError_t ie = h->f32() ? series_group_kernels_init<float>() : series_group_kernels_init<double>();
    if (ie != cudaSuccess) {
      delete h;
      return fail_cuda(ie, "series kernel attributes");
    }
    cudaGetLastError();
  }

  // ---- arena layout
  const size_t bulk = h->f32() ? sizeof(float) : sizeof(double);
  struct Item { void** ptr; size_t bytes; };
  std::vector<Item> items;
  int32_t *d_lm_seg, *d_cam_of, *d_lm_of, *d_tile_lm0, *d_tile_slot0, *d_slot_cam, *d_cam_slot_ptr, *d_cam_slot_list;
  int32_t *d_tile_desc, *d_slot_row, *d_cam_prob, *d_lm_prob, *d_tile_prob, *d_cam_off, *d_tile_off;
  uint16_t *d_meta, *d_slot_beg;
  const size_t slots = (size_t)(S.n_slots > 0 ? S.n_slots : 1);
  const size_t P = (size_t)n_probs;
  items.push_back({(void**)&d_lm_seg, sizeof(int32_t) * (nli + 1)});
  items.push_back({(void**)&d_cam_of, sizeof(int32_t) * (no > 0 ? no : 1)});
  items.push_back({(void**)&d_lm_of, sizeof(int32_t) * (no > 0 ? no : 1)});
  items.push_back({(void**)&d_meta, sizeof(uint16_t) * (no > 0 ? no : 1)});
  items.push_back({(void**)&d_tile_lm0, sizeof(int32_t) * (S.n_tiles + 1)});
  items.push_back({(void**)&d_tile_slot0, sizeof(int32_t) * (S.n_tiles + 1)});
  items.push_back({(void**)&d_tile_desc, sizeof(int32_t) * 8 * S.n_tiles});
  items.push_back({(void**)&d_slot_cam, sizeof(int32_t) * slots});
  items.push_back({(void**)&d_slot_beg, sizeof(uint16_t) * slots});
  items.push_back({(void**)&d_cam_slot_ptr, sizeof(int32_t) * (nc + 1)});
  items.push_back({(void**)&d_cam_slot_list, sizeof(int32_t) * slots});
  items.push_back({(void**)&d_slot_row, sizeof(int32_t) * slots});
  items.push_back({(void**)&d_cam_prob, sizeof(int32_t) * nc});
  items.push_back({(void**)&d_lm_prob, sizeof(int32_t) * nli});
  items.push_back({(void**)&d_tile_prob, sizeof(int32_t) * S.n_tiles});
  items.push_back({(void**)&d_cam_off, sizeof(int32_t) * (P + 1)});
  items.push_back({(void**)&d_tile_off, sizeof(int32_t) * (P + 1)});
  items.push_back({(void**)&h->obs, sizeof(double2) * (no > 0 ? no : 1)});
  if (h->weighted) items.push_back({(void**)&h->sqrt_w, sizeof(double) * (no > 0 ? no : 1)});
  items.push_back({(void**)&h->cams, sizeof(double) * nc * 9});
  items.push_back({(void**)&h->cams_trial, sizeof(double) * nc * 9});
  items.push_back({(void**)&h->lms, sizeof(double) * nli * 3});
  items.push_back({(void**)&h->prep, sizeof(double) * nc * kCamPrep});
  if (h->f32()) {
    items.push_back({(void**)&h->prep32, sizeof(float) * nc * kCamPrep});
    items.push_back({(void**)&h->obs32, sizeof(float2) * (no > 0 ? no : 1)});
    if (h->weighted) items.push_back({(void**)&h->sqrt_w32, sizeof(float) * (no > 0 ? no : 1)});
  }
  items.push_back({(void**)&h->prep_trial, sizeof(double) * nc * kCamPrep});
  items.push_back({&h->J, bulk * 24 * h->n_o_pad});
  items.push_back({&h->r, bulk * 2 * h->n_o_pad});
  items.push_back({&h->partial, bulk * kLinVals * slots});
  items.push_back({&h->t_cam, bulk * kTStride * nc});
  items.push_back({(void**)&h->U45, sizeof(double) * nc * 45});
  items.push_back({(void**)&h->b_p, sizeof(double) * nc * 9});
  items.push_back({(void**)&h->V, sizeof(double) * nli * 6});
  items.push_back({(void**)&h->b_l, sizeof(double) * nli * 3});
  items.push_back({(void**)&h->adj_p, sizeof(double) * nc * 9});
  items.push_back({(void**)&h->adj_l, sizeof(double) * nli * 3});
  items.push_back({(void**)&h->obs_caller, sizeof(int32_t) * (no > 0 ? no : 1)});
  items.push_back({(void**)&h->lm_order_dev, sizeof(int32_t) * nli});
  int32_t *d_long = nullptr, *d_lm_long = nullptr;
  if (S.n_long > 0) {
    items.push_back({(void**)&d_long, sizeof(int32_t) * 3 * S.n_long});
    items.push_back({(void**)&d_lm_long, sizeof(int32_t) * nli});
  }
  items.push_back({(void**)&h->Uinv, sizeof(double) * nc * 81});
  items.push_back({(void**)&h->Vinv, sizeof(double) * nli * 6});
  // (4 floats of slack: the staged kernel copies V^-1 ranges rounded out to 16 bytes)
  if (h->f32()) items.push_back({(void**)&h->Vinv_f, sizeof(float) * ((size_t)nli * 6 + 4)});
  items.push_back({(void**)&h->x, sizeof(double) * nc * 9});
  items.push_back({(void**)&h->dx_l, sizeof(double) * nli * 3});
  items.push_back({(void**)&h->cam_norm, sizeof(double) * 2 * nc});
  items.push_back({(void**)&h->block_cost, sizeof(double) * S.n_tiles});
  items.push_back({(void**)&h->tile_cost, sizeof(double) * S.n_tiles});
  items.push_back({(void**)&h->block_pred, sizeof(double) * S.n_tiles});
  items.push_back({(void**)&h->scalars, sizeof(double) * 4});
  items.push_back({(void**)&h->prob_cost, sizeof(double) * P});
  items.push_back({(void**)&h->gs, sizeof(GridSync)});
  uint8_t* d_tile_rec = nullptr;
  items.push_back({(void**)&d_tile_rec, S.tile_rec.size() > 0 ? S.tile_rec.size() : 16});
  items.push_back({(void**)&h->trace, sizeof(long long) * kTraceTerms * kTracePoints});
  items.push_back({(void**)&h->st, sizeof(SeriesState) * P});
  items.push_back({(void**)&h->sgl, sizeof(SeriesGlobal)});
  items.push_back({(void**)&h->rec, sizeof(LmRecord) * P});
  items.push_back({(void**)&h->not_spd, sizeof(int32_t) * P});
  items.push_back({(void**)&h->io_bad, sizeof(int32_t) * 3});
  items.push_back({(void**)&h->relin, sizeof(int32_t)});
  items.push_back({(void**)&h->chk, sizeof(CheckRecord)});
  size_t total = 0;
  for (auto& it : items) total = align_up(total, 256) + guarded(it.bytes);
  total = align_up(total, 256);

  auto bail = [&](ba_status s) { ba_destroy(h); return s; };
  cudaError_t e;
  if (descs[0].cuda_stream) {
    h->stream = (cudaStream_t)descs[0].cuda_stream;
  } else {
    e = cudaStreamCreate(&h->stream);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaStreamCreate"));
    h->own_stream = true;
  }
  e = cudaMalloc(&h->arena, total);
  if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMalloc(arena)"));
  h->arena_bytes = total;
  std::vector<uint64_t> guards;
  {
    size_t off = 0;
    for (auto& it : items) {
      off = align_up(off, 256);
      *it.ptr = (char*)h->arena + off;
      off += it.bytes;
      if (kChecks) {
        guards.push_back(off);
        off += kCanaryBytes;
      }
    }
  }
  e = cudaMemset(h->arena, 0, total);
  if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMemset(arena)"));
  e = install_canaries(h, 0, h->arena, guards);
  if (e != cudaSuccess) return bail(fail_cuda(e, "guard bytes"));
  if ((e = cudaMallocHost(&h->h_st, sizeof(SeriesState) * P)) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_sgl, sizeof(SeriesGlobal))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_rec, sizeof(LmRecord) * P)) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_gs, sizeof(GridSync))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_flag, sizeof(int32_t) * P)) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_io, sizeof(int32_t) * 3)) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_relin, sizeof(int32_t))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_scalar, sizeof(double) * 4)) != cudaSuccess)
    return bail(fail_cuda(e, "cudaMallocHost"));

  // ---- upload (sorted / internal orders)
  std::vector<double> obs_s((size_t)no * 2), sw_s;
  for (int k = 0; k < no; ++k) {
    obs_s[2 * k] = obs[2 * S.obs_order[k]];
    obs_s[2 * k + 1] = obs[2 * S.obs_order[k] + 1];
  }
  if (h->weighted) {
    sw_s.resize(no);
    for (int k = 0; k < no; ++k) sw_s[k] = std::sqrt(w[S.obs_order[k]]);
  }
  std::vector<int32_t> obs_caller((size_t)no);
  for (int k = 0; k < no; ++k) obs_caller[k] = (int32_t)S.obs_order[k];
  std::vector<double> lms_i((size_t)nli * 3);
  for (int i = 0; i < nli; ++i)
    for (int k = 0; k < 3; ++k) lms_i[i * 3 + k] = lms[(size_t)S.lm_order[i] * 3 + k];
  struct Up { void* dst; const void* src; size_t bytes; };
  std::vector<Up> ups = {
      {d_lm_seg, S.lm_seg.data(), sizeof(int32_t) * (nli + 1)},
      {d_cam_of, S.cam_of.data(), sizeof(int32_t) * no},
      {d_lm_of, S.lm_of.data(), sizeof(int32_t) * no},
      {d_meta, S.obs_meta.data(), sizeof(uint16_t) * no},
      {d_tile_lm0, S.tile_lm0.data(), sizeof(int32_t) * (S.n_tiles + 1)},
      {d_tile_slot0, S.tile_slot0.data(), sizeof(int32_t) * (S.n_tiles + 1)},
      {d_tile_desc, S.tile_desc.data(), sizeof(int32_t) * 8 * S.n_tiles},
      {d_slot_cam, S.slot_cam.data(), sizeof(int32_t) * S.n_slots},
      {d_slot_beg, S.slot_beg.data(), sizeof(uint16_t) * S.n_slots},
      {d_cam_slot_ptr, S.cam_slot_ptr.data(), sizeof(int32_t) * (nc + 1)},
      {d_cam_slot_list, S.cam_slot_list.data(), sizeof(int32_t) * S.n_slots},
      {d_slot_row, S.slot_row.data(), sizeof(int32_t) * S.n_slots},
      {d_cam_prob, S.cam_prob.data(), sizeof(int32_t) * nc},
      {d_lm_prob, S.lm_prob.data(), sizeof(int32_t) * nli},
      {d_tile_prob, tile_prob.data(), sizeof(int32_t) * S.n_tiles},
      {d_cam_off, S.cam_off.data(), sizeof(int32_t) * (P + 1)},
      {d_tile_off, S.tile_off.data(), sizeof(int32_t) * (P + 1)},
      {d_tile_rec, S.tile_rec.data(), S.tile_rec.size()},
      {h->obs, obs_s.data(), sizeof(double) * 2 * no},
      {h->obs_caller, obs_caller.data(), sizeof(int32_t) * no},
      {h->lm_order_dev, S.lm_order.data(), sizeof(int32_t) * nli},
      {h->cams, cams.data(), sizeof(double) * nc * 9},
      {h->lms, lms_i.data(), sizeof(double) * nli * 3},
  };
  std::vector<int32_t> long_tab;
  if (S.n_long > 0) {
    long_tab.insert(long_tab.end(), S.long_first.begin(), S.long_first.end());
    long_tab.insert(long_tab.end(), S.long_np.begin(), S.long_np.end());
    long_tab.insert(long_tab.end(), S.long_tile0.begin(), S.long_tile0.end());
    ups.push_back({d_long, long_tab.data(), sizeof(int32_t) * long_tab.size()});
    ups.push_back({d_lm_long, S.lm_long.data(), sizeof(int32_t) * nli});
  }
  if (h->weighted) ups.push_back({h->sqrt_w, sw_s.data(), sizeof(double) * no});
  // FP32 bulk: the observations and weights in float, rounded once here as the kernels would
  std::vector<float> obs32_s, sw32_s;
  if (h->f32()) {
    obs32_s.resize((size_t)no * 2);
    for (size_t k = 0; k < obs32_s.size(); ++k) obs32_s[k] = (float)obs_s[k];
    ups.push_back({h->obs32, obs32_s.data(), sizeof(float) * 2 * no});
    if (h->weighted) {
      sw32_s.resize(no);
      for (int k = 0; k < no; ++k) sw32_s[k] = (float)sw_s[k];
      ups.push_back({h->sqrt_w32, sw32_s.data(), sizeof(float) * no});
    }
  }
  for (auto& u : ups) {
    if (u.bytes == 0) continue;
    e = cudaMemcpy(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMemcpy(upload)"));
  }
  {
    std::vector<LmRecord> r0(P);
    for (auto& r : r0) {
      r = LmRecord{};
      r.cost = NAN;
      r.lambda = o.lambda0;
      r.nu = 2.0;
      r.active = 1;
    }
    e = cudaMemcpy(h->rec, r0.data(), sizeof(LmRecord) * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(fail_cuda(e, "cudaMemcpy(record)"));
  }

  Topology& tp = h->tp;
  tp.n_cams = nc;
  tp.n_lms = nli;
  tp.n_long = S.n_long;
  tp.long_first = d_long;
  tp.long_np = d_long ? d_long + S.n_long : nullptr;
  tp.long_tile0 = d_long ? d_long + 2 * S.n_long : nullptr;
  tp.lm_long = d_lm_long;
  tp.chk = h->chk;
  tp.n_obs = no;
  tp.n_obs_pad = h->n_o_pad;
  tp.n_tiles = S.n_tiles;
  tp.n_slots = S.n_slots;
  tp.lm_seg = d_lm_seg;
  tp.cam_of = d_cam_of;
  tp.lm_of = d_lm_of;
  tp.obs_meta = d_meta;
  tp.tile_lm0 = d_tile_lm0;
  tp.tile_slot0 = d_tile_slot0;
  tp.tile_desc = (const int4*)d_tile_desc;
  tp.slot_cam = d_slot_cam;
  tp.slot_beg = d_slot_beg;
  tp.cam_slot_ptr = d_cam_slot_ptr;
  tp.cam_slot_list = d_cam_slot_list;
  tp.slot_row = d_slot_row;
  tp.n_probs = n_probs;
  tp.cam_prob = d_cam_prob;
  tp.lm_prob = d_lm_prob;
  tp.tile_prob = d_tile_prob;
  tp.cam_off = d_cam_off;
  tp.tile_off = d_tile_off;
  tp.tile_rec = d_tile_rec;
  h->rhs_p = h->b_p;
  h->rhs_l = h->b_l;
  {
    ba_status st = rebuild_series(h, 0, kDefaultTail);
    if (st != BA_OK) return bail(st);
  }
  *out = h;
  g_last_error.clear();
  return BA_OK;
}

// Largest number of series terms any problem of the last solve used.
int max_terms(const ba_handle* h) {
  int m = 0;
  for (int p = 0; p < h->n_probs; ++p) m = h->h_st[p].m > m ? h->h_st[p].m : m;
  return m;
}

void fill_series_info(const SeriesState& S, double lambda, ba_series_info* info) {
  info->inner_iters = S.m;
  info->stopped = S.stopped;
  info->stop_value = S.stop_value;
  info->x_norm = S.x_norm;
  info->lambda = lambda;
}

void fill_step_info(const LmRecord& R, const SeriesState& S, ba_step_info* info) {
  info->cost_before = R.cost_before;
  info->cost_after = R.cost_trial;
  info->lambda = R.lambda_used;
  info->gain_ratio = R.gain_ratio;
  info->model_decrease = R.model_decrease;
  info->stop_value = S.stop_value;
  info->accepted = R.accepted;
  info->inner_iters = S.m;
  info->converged = R.converged;
  info->iteration = R.iteration - 1;
  info->not_spd = R.not_spd;
}

// The device part of one LM iteration of every problem whose record is active (batch: a
// problem that converges becomes inactive), ending with the copies of the records, the series
// states and the grid-barrier state to pinned host memory.  gated: the linearisation is gated
// on the device flag relin, which the step clears and the decision raises when a step was
// accepted (the captured form); else it runs when the host says the state moved.
ba_status seq_lm_step(ba_handle* h, bool batch, bool gated) {
  cudaStream_t s = h->stream;
  const size_t P = (size_t)h->n_probs;
  if (gated) {
    tmark(h, kTLin, 0, 0);
    launch_cam_prepare(h->cams, nullptr, h->n_c, h->prep, nullptr, s, h->prep32, h->relin);
    if (h->f32()) {
      launch_linearize<float>(h->tp, h->prep32, h->lms, h->obs32, h->sqrt_w32, (float*)h->J,
                              (float*)h->r, h->V, h->b_l, (float*)h->partial, h->block_cost, s,
                              h->relin);
      launch_lin_camera_reduce<float>(h->tp, (const float*)h->partial, h->U45, h->b_p, s,
                                      h->relin);
    } else {
      launch_linearize<double>(h->tp, h->prep, h->lms, h->obs, h->sqrt_w, (double*)h->J,
                               (double*)h->r, h->V, h->b_l, (double*)h->partial, h->block_cost,
                               s, h->relin);
      launch_lin_camera_reduce<double>(h->tp, (const double*)h->partial, h->U45, h->b_p, s,
                                       h->relin);
    }
    launch_long_track_blocks(h->tp, h->V, h->b_l, s, h->relin);
    tmark(h, kTLin, 0, 1);
    h->launches += 3 + long_kernels(h);
    CK(cudaMemsetAsync(h->relin, 0, sizeof(int32_t), s));
  } else if (!h->linearized) {
    seq_linearize(h);
  }
  ba_status st = run_solve(h, rec_field(h->rec, offsetof(LmRecord, lambda)), kRecStride, true);
  if (st != BA_OK) return st;
  Range eval_range("poba.evaluate");
  tmark(h, kTEval, 0, 0);
  launch_cam_prepare(h->cams, h->x, h->n_c, h->prep_trial, h->cams_trial, s);
  launch_tile_cost(h->tp, h->prep_trial, h->lms, h->dx_l, h->obs, h->sqrt_w, h->tile_cost, s);
  launch_lm_decide(h->tp, h->tile_cost, h->block_pred, h->not_spd, h->rec, h->opts.func_tol,
                   batch ? 1 : 0, s, gated ? h->relin : nullptr);
  launch_apply_step(h->tp, h->rec, h->cams, h->cams_trial, h->lms, h->dx_l, s);
  tmark(h, kTEval, 0, 1);
  h->launches += 4;
  st = check_launch(h, "LM step kernels");
  if (st != BA_OK) return st;
  CK(cudaMemcpyAsync(h->h_rec, h->rec, sizeof(LmRecord) * P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(SeriesState) * P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_gs, h->gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
  return BA_OK;
}

// The configuration a captured LM step depends on (besides the series schedule, whose rebuild
// drops the graph).
std::vector<double> step_key(const ba_handle* h, bool batch) {
  const ba_options& o = h->opts;
  return {o.lambda0, o.func_tol, o.eps, (double)o.max_inner, (double)o.damping_mode,
          (double)o.series_exec, (double)batch, (double)h->timing, (double)h->auto_exec,
          (double)h->plain_k, (double)h->stage_k, (double)h->flow_k,
          (double)h->barrier_timeout};
}

// Captures the device part of an LM step as a graph (once per configuration).  False: the
// capture failed (the step runs eagerly from then on).
bool capture_lm_step(ba_handle* h, bool batch) {
  const std::vector<double> key = step_key(h, batch);
  if (h->step_exec && key == h->step_key) return true;
  if (h->step_exec) {
    cudaGraphExecDestroy(h->step_exec);
    h->step_exec = nullptr;
  }
  if (h->timing && ensure_events(h) != BA_OK) return false;
  cudaStream_t s = h->stream;
  const uint64_t launches = h->launches;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->capturing = true;
  h->capturing_step = true;
  const ba_status st = seq_lm_step(h, batch, true);
  h->capturing = false;
  h->capturing_step = false;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  h->launches = launches;
  for (int c = 0; c < BA_TIMING_CLASSES; ++c) h->pending[c] = false;
  if (st != BA_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    g_last_error.clear();
    return false;
  }
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  int kernels = 0;
  for (cudaGraphNode_t n : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  e = cudaGraphInstantiate(&h->step_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->step_exec = nullptr;
    cudaGetLastError();
    return false;
  }
  h->step_kernels = kernels;
  h->step_mode = h->last_exec;
  h->step_key = key;
  return true;
}

// One LM iteration of every problem of the handle whose record is active; batch: a problem that
// converges becomes inactive.  With step graphs on (the default), the device part is one
// replay of the captured step; otherwise the same kernels launch one by one.  Reads the
// records and series states back (one synchronisation).
ba_status lm_iteration(ba_handle* h, bool batch) {
  Range range(batch ? "poba.lm_iteration_batch" : "poba.lm_iteration");
  cudaStream_t s = h->stream;
  const size_t P = (size_t)h->n_probs;
  if (!h->cost_valid) {
    seq_cost(h, rec_field(h->rec, offsetof(LmRecord, cost)), kRecStride);
    h->cost_valid = true;
  }
  h->last_solve_lm = true;
  const bool was_linearized = h->linearized;
  bool graph = h->step_graph && capture_lm_step(h, batch);
  if (h->step_graph && !graph) h->step_graph = false;  // capture unsupported: stay eager
  if (graph) {
    if (!h->relin_synced) {
      *h->h_relin = h->linearized ? 0 : 1;
      CK(cudaMemcpyAsync(h->relin, h->h_relin, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    CK(cudaGraphLaunch(h->step_exec, s));
    h->launches += (uint64_t)h->step_kernels;
    h->last_exec = h->step_mode;
    if (h->timing) {
      h->pending[kTLin] = !was_linearized;
      h->pending[kTDamp] = h->pending[kTRhs] = h->pending[kTBack] = h->pending[kTEval] = true;
    }
  } else {
    ba_status st = seq_lm_step(h, batch, false);
    if (st != BA_OK) return st;
  }
  CK(cudaStreamSynchronize(s));
  collect_timing(h, max_terms(h), true);
  if (h->last_exec >= 3 && h->h_gs->error)
    return fail(BA_ERR_TIMEOUT, "a grid barrier of the persistent series kernel timed out");
  // one linearisation covers every problem: it is stale once any problem moved
  h->linearized = true;
  for (size_t p = 0; p < P; ++p)
    if (h->h_rec[p].accepted) h->linearized = false;
  h->relin_synced = graph;  // the captured decision set relin = any step accepted
  return debug_verify(h);
}

// Status of an LM iteration after its records were read: a non-finite cost at the current state
// of an active problem.  (Blocks that were not positive definite made that problem's step a
// rejected one; its step info says so.)
ba_status lm_status(ba_handle* h) {
  for (int p = 0; p < h->n_probs; ++p)
    if (!std::isfinite(h->h_rec[p].cost_before))
      return fail(BA_ERR_NONFINITE, h->n_probs > 1 ? "problem " + std::to_string(p) +
                                                         ": non-finite cost at the current state"
                                                   : std::string("non-finite cost at the current state"));
  return BA_OK;
}

}  // namespace

extern "C" {

ba_status ba_create(const ba_problem_desc* d, const ba_options* opts, ba_handle** out) {
  return create_impl(d, 1, opts, out);
}

ba_status ba_create_batch(const ba_problem_desc* descs, int32_t n_problems, const ba_options* opts,
                          ba_handle** out) {
  return create_impl(descs, n_problems, opts, out);
}

ba_status ba_get_batch_layout(ba_handle* h, int32_t* n_problems, int32_t* cam_off, int32_t* lm_off) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (n_problems) *n_problems = h->n_probs;
  if (cam_off) std::memcpy(cam_off, h->cam_off_h.data(), sizeof(int32_t) * (h->n_probs + 1));
  if (lm_off) std::memcpy(lm_off, h->lm_off_h.data(), sizeof(int32_t) * (h->n_probs + 1));
  return BA_OK;
}

ba_status ba_set_options(ba_handle* h, const ba_options* o) {
  if (!h || !o) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  std::string why;
  if (!valid_options(*o, &why)) return fail(BA_ERR_INVALID_ARG, why);
  h->opts = *o;
  return BA_OK;
}

ba_status ba_linearize(ba_handle* h, double* cost_out) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  seq_linearize(h);
  ba_status st = check_launch(h, "linearize kernels");
  if (st != BA_OK) return st;
  h->linearized = true;
  h->relin_synced = false;
  if (cost_out) {
    launch_reduce_sum(h->block_cost, h->tp.n_tiles, h->scalars + 1, 1.0, h->stream);
    h->launches += 1;
    CK(cudaMemcpyAsync(h->h_scalar, h->scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *cost_out = h->h_scalar[0];
  }
  return BA_OK;
}

ba_status ba_solve_schur_power(ba_handle* h, double lambda, ba_series_info* info) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!h->linearized) return fail(BA_ERR_NOT_LINEARIZED, "ba_linearize has not been called");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(BA_ERR_INVALID_ARG, "lambda must be finite and > 0");
  launch_set_scalar(h->scalars + 0, lambda, h->stream);
  h->launches += 1;
  h->solve_lambda = lambda;
  h->last_solve_lm = false;
  ba_status st = run_solve(h, h->scalars + 0, 0, false);
  if (st != BA_OK) return st;
  if (!info) return BA_OK;
  const size_t P = (size_t)h->n_probs;
  CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(SeriesState) * P, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_flag, h->not_spd, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_gs, h->gs, sizeof(GridSync), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  collect_timing(h, max_terms(h), true);
  if (h->last_exec >= 3 && h->h_gs->error)
    return fail(BA_ERR_TIMEOUT, "a grid barrier of the persistent series kernel timed out");
  if (P == 1) {
    fill_series_info(h->h_st[0], lambda, info);
  } else {
    // a batch: the largest term count and stop value, stopped iff every problem stopped, and
    // the norm of the whole camera step
    ba_series_info a{};
    a.stopped = 1;
    a.stop_value = -INFINITY;
    double x2 = 0.0;
    for (size_t p = 0; p < P; ++p) {
      const SeriesState& S = h->h_st[p];
      a.inner_iters = S.m > a.inner_iters ? S.m : a.inner_iters;
      a.stopped = a.stopped && S.stopped;
      a.stop_value = S.stop_value > a.stop_value ? S.stop_value : a.stop_value;
      x2 += S.x_norm * S.x_norm;
    }
    a.x_norm = std::sqrt(x2);
    a.lambda = lambda;
    *info = a;
  }
  for (size_t p = 0; p < P; ++p)
    if (h->h_flag[p])
      return fail(BA_ERR_NOT_SPD, P > 1 ? "problem " + std::to_string(p) +
                                              ": a damped block is not positive definite"
                                        : std::string("a damped block is not positive definite"));
  return BA_OK;
}

ba_status ba_autotune(ba_handle* h, int32_t trials, int32_t* exec_out, int32_t* bps_out) {
  Range range("poba.autotune");
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (trials < 1) return fail(BA_ERR_INVALID_ARG, "trials must be >= 1");
  if (!h->linearized) {
    seq_linearize(h);
    ba_status st = check_launch(h, "linearize kernels");
    if (st != BA_OK) return st;
    h->linearized = true;
    h->relin_synced = false;
  }
  // a candidate: execution form, blocks per SM, group size
  struct Cand {
    int exec, k, target, tail;
  };
  const ba_options saved = h->opts;
  const bool saved_timing = h->timing;
  const int saved_k = h->plain_k, saved_sk = h->stage_k, saved_fk = h->flow_k,
            saved_target = h->ser.target,
            saved_req = h->group_obs, saved_tail = h->ser.tail;
  h->opts.eps = 0.0;  // every candidate runs max_inner terms
  h->timing = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ba_status st = BA_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = fail_cuda(cudaGetLastError(), "cudaEventCreate");
  launch_set_scalar(h->scalars + 0, h->opts.lambda0, h->stream);
  h->launches += 1;
  h->last_solve_lm = false;
  h->solve_lambda = h->opts.lambda0;
  float best_ms = 0.f;
  Cand best{-1, 0, 0, 0};
  auto trial = [&](const Cand& c) {
    if (st != BA_OK) return;
    if ((c.target != h->ser.target || c.tail != h->ser.tail) &&
        (st = rebuild_series(h, c.target, c.tail)) != BA_OK)
      return;
    h->opts.series_exec = c.exec;
    if (c.exec == 3) h->plain_k = c.k;
    if (c.exec == 4) h->stage_k = c.k;
    if (c.exec == 5) h->flow_k = c.k;
    st = run_solve(h, h->scalars + 0, 0, false);  // warm-up (and graph capture)
    if (st != BA_OK) return;
    cudaEventRecord(e0, h->stream);
    for (int t = 0; t < trials && st == BA_OK; ++t) st = run_solve(h, h->scalars + 0, 0, false);
    cudaEventRecord(e1, h->stream);
    if (st != BA_OK) return;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = fail_cuda(e, "autotune");
      return;
    }
    e = cudaMemcpy(h->h_gs, h->gs, sizeof(GridSync), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      st = fail_cuda(e, "autotune");
      return;
    }
    if (c.exec >= 3 && h->h_gs->error) {
      st = fail(BA_ERR_TIMEOUT, "a grid barrier of the persistent series kernel timed out");
      return;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best.exec < 0 || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  };
  // the persistent kernel at each residency with one group per block; then two groups per
  // block at the best residency (finer load balance, more partial rows); then the per-term
  // launches replayed as a graph on the best schedule
  for (int k = 1; k <= h->plain_max; ++k)
    trial({3, k, series_auto_target(h->n_o, auto_groups(h, k * h->sms - 1)), kDefaultTail});
  for (int k = 1; k <= h->stage_max && !has_long_groups(h); ++k)
    trial({4, k, series_auto_target(h->n_o, auto_groups(h, k * h->sms - 1)), kDefaultTail});
  for (int k = 1; k <= h->flow_max && !has_long_groups(h); ++k)
    trial({5, k, series_auto_target(h->n_o, auto_groups(h, k * h->sms)), kDefaultTail});
  if (best.exec >= 3) {
    const Cand b = best;
    trial({b.exec, b.k, b.target, 0});
    trial({b.exec, b.k, b.target, 4});
    if (b.target > kChunkObs) trial({b.exec, b.k, (b.target + 1) / 2, b.tail});
  }
  trial({1, 0, best.exec < 0 ? h->ser.target : best.target, best.exec < 0 ? h->ser.tail : best.tail});
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  h->opts = saved;
  h->timing = saved_timing;
  h->plain_k = saved_k;
  h->stage_k = saved_sk;
  h->flow_k = saved_fk;
  if (st != BA_OK) {
    if (h->ser.target != saved_target || h->ser.tail != saved_tail)
      rebuild_series(h, saved_req, saved_tail);
    return st;
  }
  if (best.target != h->ser.target || best.tail != h->ser.tail) {
    st = rebuild_series(h, best.target, best.tail);
    if (st != BA_OK) return st;
  }
  h->group_obs = best.target;
  h->auto_exec = best.exec;
  if (best.exec == 3) h->plain_k = best.k;
  if (best.exec == 4) h->stage_k = best.k;
  if (best.exec == 5) h->flow_k = best.k;
  if (exec_out) *exec_out = best.exec;
  if (bps_out) *bps_out = best.exec >= 3 ? best.k : 0;
  return BA_OK;
}

ba_status ba_set_step_graph(ba_handle* h, int32_t enable) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  h->step_graph = enable != 0;
  return BA_OK;
}

ba_status ba_get_step_graph(ba_handle* h, int32_t* enabled, int32_t* kernels_per_step) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (enabled) *enabled = h->step_graph ? 1 : 0;
  if (kernels_per_step) *kernels_per_step = h->step_exec ? h->step_kernels : 0;
  return BA_OK;
}

ba_status ba_get_schedule(ba_handle* h, ba_schedule* out) {
  if (!h || !out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  out->group_obs = h->ser.target;
  out->tail_parts = h->ser.tail;
  out->series_exec = h->auto_exec;
  out->blocks_per_sm = h->auto_exec == 4 ? h->stage_k : h->auto_exec == 5 ? h->flow_k : h->plain_k;
  out->n_groups = h->ser.n_groups;
  out->n_chunks = h->ser.n_chunks;
  out->n_group_slots = h->ser.n_gslots;
  return BA_OK;
}

ba_status ba_set_schedule(ba_handle* h, const ba_schedule* in) {
  if (!h || !in) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  if (in->group_obs < 0) return fail(BA_ERR_INVALID_ARG, "group_obs must be >= 0");
  if (in->tail_parts < 0 || in->tail_parts > 64)
    return fail(BA_ERR_INVALID_ARG, "tail_parts must be in [0, 64]");
  if (in->series_exec != 1 && in->series_exec != 3 && in->series_exec != 4 &&
      in->series_exec != 5)
    return fail(BA_ERR_INVALID_ARG, "series_exec must be 1, 3, 4 or 5");
  if (in->series_exec == 4 && h->stage_max <= 0)
    return fail(BA_ERR_INVALID_ARG, "series_exec 4 needs BA_FP32_BULK and the staged kernel");
  if (in->series_exec == 5 && h->flow_max <= 0)
    return fail(BA_ERR_INVALID_ARG, "series_exec 5 needs the dataflow kernel (cooperative launch)");
  if ((in->series_exec == 4 || in->series_exec == 5) && has_long_groups(h))
    return fail(BA_ERR_INVALID_ARG,
                "series_exec 4 and 5 take no tracks of more than 256 observations (nor, in FP64, "
                "landmarks seen by more than 96 cameras)");
  const int kmax = in->series_exec == 4 ? h->stage_max : in->series_exec == 5 ? h->flow_max
                                                                              : h->plain_max;
  if (in->series_exec >= 3 && (in->blocks_per_sm < 1 || in->blocks_per_sm > kmax))
    return fail(BA_ERR_INVALID_ARG, "blocks_per_sm must be in [1, " + std::to_string(kmax) +
                                        "] (the persistent kernel's residency on this device)");
  const int target = in->group_obs > 0 ? in->group_obs : series_auto_target(h->n_o, auto_workers(h));
  if (target != h->ser.target || in->tail_parts != h->ser.tail) {
    ba_status st = rebuild_series(h, in->group_obs, in->tail_parts);
    if (st != BA_OK) return st;
  }
  h->group_obs = in->group_obs;
  h->auto_exec = in->series_exec;
  if (in->series_exec == 3) h->plain_k = in->blocks_per_sm;
  if (in->series_exec == 4) h->stage_k = in->blocks_per_sm;
  if (in->series_exec == 5) h->flow_k = in->blocks_per_sm;
  return BA_OK;
}

ba_status ba_adjoint(ba_handle* h, double lambda, const double* g_cams, const double* g_lms,
                     double* d_obs, double* d_weights, int32_t ptr_kind, ba_series_info* info) {
  Range range("poba.adjoint");
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(BA_ERR_INVALID_ARG, "lambda must be finite and > 0");
  if (!g_cams || !g_lms || !d_obs) return fail(BA_ERR_INVALID_ARG, "g_cams / g_lms / d_obs is NULL");
  if (ptr_kind != 0 && ptr_kind != 1) return fail(BA_ERR_INVALID_ARG, "ptr_kind must be 0 or 1");
  cudaStream_t s = h->stream;
  const size_t nc9 = (size_t)h->n_c * 9, nl3 = (size_t)h->n_l * 3, no = (size_t)h->n_o;
  if (!h->linearized) {
    seq_linearize(h);
    ba_status st = check_launch(h, "linearize kernels");
    if (st != BA_OK) return st;
    h->linearized = true;
    h->relin_synced = false;
  }
  // the incoming gradient: device inputs are read in place, host inputs are staged in the
  // step buffers (which the solve overwrites)
  const double* gp = g_cams;
  const double* gl = g_lms;
  if (ptr_kind == 0) {
    CK(cudaMemcpyAsync(h->x, g_cams, sizeof(double) * nc9, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->dx_l, g_lms, sizeof(double) * nl3, cudaMemcpyHostToDevice, s));
    gp = h->x;
    gl = h->dx_l;
  }
  launch_adjoint_rhs(h->n_c, h->n_li, h->lm_order_dev, gp, gl, h->adj_p, h->adj_l, s);
  launch_set_scalar(h->scalars + 0, lambda, s);
  h->launches += 2;
  h->solve_lambda = lambda;
  h->last_solve_lm = false;
  h->rhs_p = h->adj_p;
  h->rhs_l = h->adj_l;
  ba_status st = run_solve(h, h->scalars + 0, 0, false);
  h->rhs_p = h->b_p;
  h->rhs_l = h->b_l;
  if (st != BA_OK) return st;
  // a = (x, dx_l); per-observation gradients in the caller's order
  double* out_obs = d_obs;
  double* out_w = d_weights;
  if (ptr_kind == 0) {
    if (!h->grad_out) {
      cudaError_t e = cudaMalloc(&h->grad_out, sizeof(double) * 3 * (no > 0 ? no : 1));
      if (e != cudaSuccess) return fail_cuda(e, "cudaMalloc(adjoint outputs)");
    }
    out_obs = h->grad_out;
    out_w = d_weights ? h->grad_out + 2 * no : nullptr;
  }
  if (h->f32())
    launch_obs_gradient<float>(h->tp, (const float*)h->J, (const float*)h->r, h->sqrt_w, h->x,
                               h->dx_l, h->obs_caller, out_obs, out_w, s);
  else
    launch_obs_gradient<double>(h->tp, (const double*)h->J, (const double*)h->r, h->sqrt_w,
                                h->x, h->dx_l, h->obs_caller, out_obs, out_w, s);
  h->launches += no > 0 ? 1 : 0;
  st = check_launch(h, "adjoint gradient kernel");
  if (st != BA_OK) return st;
  if (ptr_kind == 0 && no > 0) {
    CK(cudaMemcpyAsync(d_obs, out_obs, sizeof(double) * 2 * no, cudaMemcpyDeviceToHost, s));
    if (d_weights) CK(cudaMemcpyAsync(d_weights, out_w, sizeof(double) * no, cudaMemcpyDeviceToHost, s));
  }
  const size_t P = (size_t)h->n_probs;
  CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(SeriesState) * P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_flag, h->not_spd, sizeof(int32_t) * P, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->h_gs, h->gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  collect_timing(h, max_terms(h), true);
  if (h->last_exec >= 3 && h->h_gs->error)
    return fail(BA_ERR_TIMEOUT, "a grid barrier of the persistent series kernel timed out");
  if (info) {
    int m = 0, stopped = 1;
    double sv = -INFINITY, x2 = 0.0;
    for (size_t p = 0; p < P; ++p) {
      const SeriesState& S = h->h_st[p];
      m = S.m > m ? S.m : m;
      stopped = stopped && S.stopped;
      sv = S.stop_value > sv ? S.stop_value : sv;
      x2 += S.x_norm * S.x_norm;
    }
    info->inner_iters = m;
    info->stopped = stopped;
    info->stop_value = P == 1 ? h->h_st[0].stop_value : sv;
    info->x_norm = P == 1 ? h->h_st[0].x_norm : std::sqrt(x2);
    info->lambda = lambda;
  }
  for (size_t p = 0; p < P; ++p)
    if (h->h_flag[p]) return fail(BA_ERR_NOT_SPD, "a damped block is not positive definite");
  return BA_OK;
}

}  // extern "C"

namespace {

ba_status ensure_pcg(ba_handle* h) {
  if (h->pcg) return BA_OK;
  const size_t n9 = (size_t)h->n_c * 9, n45 = (size_t)h->n_c * 45, n81 = (size_t)h->n_c * 81;
  const size_t total = 6 * n9 + kPcgCount + kPcgDotBlocks + 2 * n45 + n81;
  CK(cudaMalloc(&h->pcg, sizeof(double) * total));
  double* q = h->pcg;
  double** bufs[] = {&h->pcg_y, &h->pcg_r, &h->pcg_z, &h->pcg_p, &h->pcg_q, &h->pcg_rhs};
  for (double** b : bufs) {
    *b = q;
    q += n9;
  }
  h->pcg_sc = q;
  q += kPcgCount;
  h->pcg_part = q;
  q += kPcgDotBlocks;
  h->pcg_sj = q;
  q += n45;
  h->pcg_s45 = q;
  q += n45;
  h->pcg_minv = q;
  CK(cudaMemsetAsync(h->pcg_sc, 0, sizeof(double) * kPcgCount, h->stream));
  return BA_OK;
}

// S p (float64 p, q): stage p as the series term, W V^-1 W^T p in the tiles, U_lam p - y per
// camera.
template <typename T>
void seq_schur_apply(ba_handle* h, double lambda, const double* p, double* q) {
  cudaStream_t s = h->stream;
  const T* Vi = h->f32() ? (const T*)(const void*)h->Vinv_f : (const T*)(const void*)h->Vinv;
  launch_stage_term<T>(h->n_c, p, (T*)h->t_cam, s);
  launch_series_reset(h->st, h->sgl, nullptr, h->n_probs, s);
  launch_tile_series<T>(h->tp, h->sp, (const T*)h->J, (const T*)h->t_cam, Vi,
                        (T*)h->ser_partial, h->st, h->sgl, s);
  launch_schur_camera<T>(h->tp, h->sp, (const T*)h->ser_partial, h->U45, lambda,
                         h->opts.damping_mode, p, q, s);
  h->launches += 3 + (h->sp.n_groups > 0 ? 1 : 0);
}

// The reduced right-hand side -b~ = W V^-1 b_l - b_p.
template <typename T>
void seq_schur_rhs(ba_handle* h, double* out) {
  cudaStream_t s = h->stream;
  const T* Vi = h->f32() ? (const T*)(const void*)h->Vinv_f : (const T*)(const void*)h->Vinv;
  launch_series_reset(h->st, h->sgl, nullptr, h->n_probs, s);
  launch_tile_rhs<T>(h->tp, h->sp, (const T*)h->J, h->b_l, Vi, (T*)h->ser_partial, h->st, s);
  launch_schur_rhs_camera<T>(h->tp, h->sp, (const T*)h->ser_partial, h->b_p, out, s);
  h->launches += 2 + (h->sp.n_groups > 0 ? 1 : 0);
}

// Schur-Jacobi blocks S_cc and their inverses.
template <typename T>
void seq_schur_jacobi(ba_handle* h, double lambda) {
  cudaStream_t s = h->stream;
  launch_schur_jacobi_tiles<T>(h->tp, (const T*)h->J, h->Vinv, (T*)h->partial, s);
  launch_lin_camera_reduce<T>(h->tp, (const T*)h->partial, h->pcg_sj, h->pcg_z, s);
  launch_schur_diag(h->n_c, h->U45, h->pcg_sj, lambda, h->opts.damping_mode, h->pcg_s45, s);
  launch_invert_camera_blocks(h->tp, h->pcg_s45, h->pcg_sc + kPcgZero, h->opts.damping_mode,
                              h->pcg_minv, h->not_spd, s);
  h->launches += 4;
}

// z = M^-1 r.  Power series: the series solve with the right-hand side (b_p, b_l) = (-r, 0),
// i.e. x(m) = sum_{i<=m} P^i U^-1 r.
ba_status precondition(ba_handle* h, int precond, int m, const double* r, double* z) {
  cudaStream_t s = h->stream;
  if (precond == 0) {
    launch_block_apply(h->n_c, h->pcg_minv, r, z, s);
    h->launches += 1;
    return BA_OK;
  }
  launch_negate(h->n_c * 9, r, h->adj_p, s);
  CK(cudaMemsetAsync(h->adj_l, 0, sizeof(double) * (size_t)h->n_li * 3, s));
  const ba_options saved = h->opts;
  h->opts.eps = 0.0;
  h->opts.max_inner = m;
  h->rhs_p = h->adj_p;
  h->rhs_l = h->adj_l;
  ba_status st = run_series_body(h, false);
  h->rhs_p = h->b_p;
  h->rhs_l = h->b_l;
  h->opts = saved;
  if (st != BA_OK) return st;
  CK(cudaMemcpyAsync(z, h->x, sizeof(double) * (size_t)h->n_c * 9, cudaMemcpyDeviceToDevice, s));
  h->launches += 1;
  return BA_OK;
}

template <typename T>
ba_status pcg_solve(ba_handle* h, double lambda, int precond, int m, double rtol, int max_iter,
                    ba_pcg_info* info) {
  cudaStream_t s = h->stream;
  const int n = h->n_c * 9;
  seq_schur_rhs<T>(h, h->pcg_rhs);
  if (precond == 0) seq_schur_jacobi<T>(h, lambda);
  CK(cudaMemsetAsync(h->pcg_y, 0, sizeof(double) * n, s));
  CK(cudaMemcpyAsync(h->pcg_r, h->pcg_rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  launch_dot(n, h->pcg_rhs, h->pcg_rhs, h->pcg_part, h->pcg_sc + kPcgBb, s);
  ba_status st = precondition(h, precond, m, h->pcg_r, h->pcg_z);
  if (st != BA_OK) return st;
  launch_dot(n, h->pcg_r, h->pcg_z, h->pcg_part, h->pcg_sc + kPcgRzNew, s);
  launch_cg_direction(n, h->pcg_sc, h->pcg_z, h->pcg_p, 1, s);
  h->launches += 6;
  int it = 0;
  double rel = 1.0, bb = 0.0;
  bool conv = false;
  for (it = 1; it <= max_iter; ++it) {
    seq_schur_apply<T>(h, lambda, h->pcg_p, h->pcg_q);
    launch_dot(n, h->pcg_p, h->pcg_q, h->pcg_part, h->pcg_sc + kPcgPq, s);
    launch_cg_update(n, h->pcg_sc, h->pcg_p, h->pcg_q, h->pcg_y, h->pcg_r, s);
    launch_dot(n, h->pcg_r, h->pcg_r, h->pcg_part, h->pcg_sc + kPcgRr, s);
    h->launches += 5;
    CK(cudaMemcpyAsync(h->h_scalar, h->pcg_sc + kPcgRr, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    st = check_launch(h, "PCG kernels");
    if (st != BA_OK) return st;
    bb = h->h_scalar[1];
    rel = bb > 0.0 ? std::sqrt(h->h_scalar[0] / bb) : 0.0;
    if (!std::isfinite(rel)) return fail(BA_ERR_NONFINITE, "non-finite PCG residual");
    if (rel <= rtol) {
      conv = true;
      break;
    }
    if (it == max_iter) break;
    st = precondition(h, precond, m, h->pcg_r, h->pcg_z);
    if (st != BA_OK) return st;
    launch_dot(n, h->pcg_r, h->pcg_z, h->pcg_part, h->pcg_sc + kPcgRzNew, s);
    launch_cg_direction(n, h->pcg_sc, h->pcg_z, h->pcg_p, 0, s);
    h->launches += 4;
  }
  if (bb == 0.0) {
    rel = 0.0;
    conv = true;
  }
  // dx_p = y, dx_l by back-substitution
  CK(cudaMemcpyAsync(h->x, h->pcg_y, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  const T* Vi = h->f32() ? (const T*)(const void*)h->Vinv_f : (const T*)(const void*)h->Vinv;
  launch_tile_backsub<T>(h->tp, (const T*)h->J, (const T*)h->r, h->x, h->b_l, Vi, h->dx_l,
                         h->block_pred, s);
  h->launches += 1 + long_kernels(h);
  CK(cudaMemcpyAsync(h->h_flag, h->not_spd, sizeof(int32_t) * h->n_probs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  st = check_launch(h, "PCG back-substitution");
  if (st != BA_OK) return st;
  h->have_step = true;
  if (info) {
    info->iterations = it > max_iter ? max_iter : it;
    info->converged = conv ? 1 : 0;
    info->rel_residual = rel;
    info->lambda = lambda;
  }
  for (int p = 0; p < h->n_probs; ++p)
    if (h->h_flag[p]) return fail(BA_ERR_NOT_SPD, "a damped block is not positive definite");
  return BA_OK;
}

}  // namespace

extern "C" {

ba_status ba_solve_schur_pcg(ba_handle* h, double lambda, int32_t precond, int32_t m_precond,
                             double rtol, int32_t max_iter, ba_pcg_info* info) {
  Range range("poba.pcg");
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!h->linearized) return fail(BA_ERR_NOT_LINEARIZED, "ba_linearize has not been called");
  if (!(lambda > 0.0) || !std::isfinite(lambda)) return fail(BA_ERR_INVALID_ARG, "lambda must be finite and > 0");
  if (precond != 0 && precond != 1) return fail(BA_ERR_INVALID_ARG, "precond must be 0 (Schur-Jacobi) or 1 (power series)");
  if (m_precond < 0 || m_precond > 10000) return fail(BA_ERR_INVALID_ARG, "m_precond out of range [0, 10000]");
  if (!(rtol >= 0.0) || max_iter < 1) return fail(BA_ERR_INVALID_ARG, "need rtol >= 0 and max_iter >= 1");
  ba_status st = ensure_pcg(h);
  if (st != BA_OK) return st;
  CK(cudaMemsetAsync(h->not_spd, 0, sizeof(int32_t) * h->n_probs, h->stream));
  launch_set_scalar(h->scalars + 0, lambda, h->stream);
  launch_damp_invert(h->tp, h->U45, h->V, h->scalars + 0, 0, h->opts.damping_mode, h->Uinv,
                     h->Vinv, h->f32() ? h->Vinv_f : nullptr, h->not_spd, h->stream);
  h->launches += 2;
  h->solve_lambda = lambda;
  h->last_solve_lm = false;
  return h->f32() ? pcg_solve<float>(h, lambda, precond, m_precond, rtol, max_iter, info)
                  : pcg_solve<double>(h, lambda, precond, m_precond, rtol, max_iter, info);
}

ba_status ba_get_series_state(ba_handle* h, ba_series_info* infos) {
  if (!h || !infos) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  const size_t P = (size_t)h->n_probs;
  CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(SeriesState) * P, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_rec, h->rec, sizeof(LmRecord) * P, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t p = 0; p < P; ++p)
    fill_series_info(h->h_st[p], h->last_solve_lm ? h->h_rec[p].lambda_used : h->solve_lambda, &infos[p]);
  return BA_OK;
}

ba_status ba_lm_step(ba_handle* h, ba_step_info* info) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (h->n_probs != 1) return fail(BA_ERR_INVALID_ARG, "a batch handle steps with ba_lm_step_batch");
  ba_status st = lm_iteration(h, false);
  if (st != BA_OK) return st;
  if (info) fill_step_info(h->h_rec[0], h->h_st[0], info);
  return lm_status(h);
}

ba_status ba_lm_solve(ba_handle* h, ba_step_info* trace, int32_t* n_steps) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (h->n_probs != 1) return fail(BA_ERR_INVALID_ARG, "a batch handle solves with ba_lm_solve_batch");
  int n = 0;
  ba_status st = BA_OK;
  for (int it = 0; it < h->opts.max_lm; ++it) {
    ba_step_info si{};
    st = ba_lm_step(h, &si);
    if (trace) trace[n] = si;
    ++n;
    if (st != BA_OK || si.converged) break;
  }
  if (n_steps) *n_steps = n;
  return st;
}

ba_status ba_lm_step_batch(ba_handle* h, ba_step_info* infos, int32_t* n_active) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  ba_status st = lm_iteration(h, true);
  if (st != BA_OK) return st;
  int active = 0;
  for (int p = 0; p < h->n_probs; ++p) {
    if (infos) fill_step_info(h->h_rec[p], h->h_st[p], &infos[p]);
    active += h->h_rec[p].active ? 1 : 0;
  }
  if (n_active) *n_active = active;
  return lm_status(h);
}

ba_status ba_lm_solve_batch(ba_handle* h, ba_step_info* infos, int32_t* n_steps) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  int n = 0;
  ba_status st = BA_OK;
  for (int it = 0; it < h->opts.max_lm; ++it) {
    int32_t active = 0;
    st = ba_lm_step_batch(h, infos, &active);
    ++n;
    if (st != BA_OK || active == 0) break;
  }
  if (n_steps) *n_steps = n;
  return st;
}

ba_status ba_cost(ba_handle* h, double* cost_out) {
  Range range("poba.cost");
  if (!h || !cost_out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  launch_cam_prepare(h->cams, nullptr, h->n_c, h->prep, nullptr, h->stream);
  launch_tile_cost(h->tp, h->prep, h->lms, nullptr, h->obs, h->sqrt_w, h->tile_cost, h->stream);
  launch_reduce_sum(h->tile_cost, h->tp.n_tiles, h->scalars + 1, 0.5, h->stream);
  h->launches += 3;
  ba_status st = check_launch(h, "cost kernels");
  if (st != BA_OK) return st;
  CK(cudaMemcpyAsync(h->h_scalar, h->scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *cost_out = h->h_scalar[0];
  return BA_OK;
}

ba_status ba_cost_batch(ba_handle* h, double* costs) {
  if (!h || !costs) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  seq_cost(h, h->prob_cost, 1);
  ba_status st = check_launch(h, "cost kernels");
  if (st != BA_OK) return st;
  CK(cudaMemcpyAsync(costs, h->prob_cost, sizeof(double) * h->n_probs, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BA_OK;
}

}  // extern "C"

namespace {

// Camera [n_c][9] and landmark [n_l][3] arrays out in the caller's order (landmarks permuted on
// the device through the staging buffer adj_l); one synchronisation.
ba_status state_out(ba_handle* h, const double* cams_dev, const double* lms_dev, double* cams,
                    double* lms, int32_t ptr_kind) {
  if (ptr_kind != 0 && ptr_kind != 1) return fail(BA_ERR_INVALID_ARG, "ptr_kind must be 0 or 1");
  cudaStream_t s = h->stream;
  const cudaMemcpyKind kind = ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cams) CK(cudaMemcpyAsync(cams, cams_dev, sizeof(double) * (size_t)h->n_c * 9, kind, s));
  if (lms) {
    // every piece of a long track holds the same values: its copies land on one caller row
    launch_scatter_rows3(lms_dev, h->lm_order_dev, h->n_li, h->adj_l, s);
    h->launches += 1;
    CK(cudaMemcpyAsync(lms, h->adj_l, sizeof(double) * (size_t)h->n_l * 3, kind, s));
  }
  CK(cudaStreamSynchronize(s));
  return check_launch(h, "state output");
}

}  // namespace

extern "C" {

ba_status ba_get_params(ba_handle* h, double* cams, double* lms, int32_t ptr_kind) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  return state_out(h, h->cams, h->lms, cams, lms, ptr_kind);
}

ba_status ba_set_params(ba_handle* h, const double* cams, const double* lms, int32_t ptr_kind) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (ptr_kind != 0 && ptr_kind != 1) return fail(BA_ERR_INVALID_ARG, "ptr_kind must be 0 or 1");
  cudaStream_t s = h->stream;
  const size_t nc9 = (size_t)h->n_c * 9, nl3 = (size_t)h->n_l * 3;
  // host inputs are copied into the staging buffers first; the state changes only once every
  // value is known to be finite
  const double* c_src = cams;
  const double* l_src = lms;
  if (ptr_kind == 0) {
    if (cams) CK(cudaMemcpyAsync(h->adj_p, cams, sizeof(double) * nc9, cudaMemcpyHostToDevice, s));
    if (lms) CK(cudaMemcpyAsync(h->adj_l, lms, sizeof(double) * nl3, cudaMemcpyHostToDevice, s));
    c_src = h->adj_p;
    l_src = h->adj_l;
  }
  CK(cudaMemsetAsync(h->io_bad, 0, sizeof(int32_t) * 3, s));
  if (cams) launch_check_finite(c_src, (int)nc9, h->io_bad + 0, s);
  if (lms) launch_check_finite(l_src, (int)nl3, h->io_bad + 1, s);
  // a state equal to the current one in every bit (typically the state a rejected LM step
  // left, read back and passed in again) keeps the linearisation and the cost
  if (cams) launch_state_differs(c_src, h->cams, nullptr, (int)nc9, h->io_bad + 2, s);
  if (lms) launch_state_differs(l_src, h->lms, h->lm_order_dev, h->n_li, h->io_bad + 2, s);
  h->launches += (cams ? 2 : 0) + (lms ? 2 : 0);
  CK(cudaMemcpyAsync(h->h_io, h->io_bad, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  ba_status st = check_launch(h, "state input");
  if (st != BA_OK) return st;
  if (h->h_io[0]) return fail(BA_ERR_NONFINITE, "non-finite camera parameter");
  if (h->h_io[1]) return fail(BA_ERR_NONFINITE, "non-finite landmark");
  if (!h->h_io[2]) return BA_OK;
  if (cams) CK(cudaMemcpyAsync(h->cams, c_src, sizeof(double) * nc9, cudaMemcpyDeviceToDevice, s));
  if (lms) launch_gather_rows3(l_src, h->lm_order_dev, h->n_li, h->lms, s);
  h->launches += lms ? 1 : 0;
  h->linearized = false;
  h->relin_synced = false;
  h->cost_valid = false;
  return check_launch(h, "state input");
}

ba_status ba_get_step(ba_handle* h, double* dx_p, double* dx_l, int32_t ptr_kind) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  return state_out(h, h->x, h->dx_l, dx_p, dx_l, ptr_kind);
}

ba_status ba_get_linearization(ba_handle* h, double* r, double* Jp, double* Jl, int32_t ptr_kind) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!h->linearized) return fail(BA_ERR_NOT_LINEARIZED, "no current linearisation");
  if (ptr_kind != 0 && ptr_kind != 1) return fail(BA_ERR_INVALID_ARG, "ptr_kind must be 0 or 1");
  CK(cudaStreamSynchronize(h->stream));
  const size_t pad = (size_t)h->n_o_pad, no = (size_t)h->n_o;
  std::vector<double> Jd(24 * pad), rd(2 * pad);
  if (h->f32()) {
    std::vector<float> Jf(24 * pad), rf(2 * pad);
    CK(cudaMemcpy(Jf.data(), h->J, sizeof(float) * Jf.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rf.data(), h->r, sizeof(float) * rf.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < Jf.size(); ++i) Jd[i] = Jf[i];
    for (size_t i = 0; i < rf.size(); ++i) rd[i] = rf[i];
  } else {
    CK(cudaMemcpy(Jd.data(), h->J, sizeof(double) * Jd.size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rd.data(), h->r, sizeof(double) * rd.size(), cudaMemcpyDeviceToHost));
  }
  std::vector<double> ro(no * 2), jpo(no * 18), jlo(no * 6);
  for (size_t o = 0; o < no; ++o) {
    const size_t c = (size_t)h->sched.obs_order[o];
    for (int i = 0; i < 2; ++i) ro[c * 2 + i] = rd[i * pad + o];
    const bool f32 = h->f32();
    for (int p = 0; p < 18; ++p)
      jpo[c * 18 + p] = Jd[f32 ? jidx<float>(p, o, pad) : jidx<double>(p, o, pad)];
    for (int p = 0; p < 6; ++p)
      jlo[c * 6 + p] = Jd[f32 ? jidx<float>(18 + p, o, pad) : jidx<double>(18 + p, o, pad)];
  }
  ba_status st;
  if (r && (st = copy_out(r, ro.data(), sizeof(double) * ro.size(), ptr_kind)) != BA_OK) return st;
  if (Jp && (st = copy_out(Jp, jpo.data(), sizeof(double) * jpo.size(), ptr_kind)) != BA_OK) return st;
  if (Jl && (st = copy_out(Jl, jlo.data(), sizeof(double) * jlo.size(), ptr_kind)) != BA_OK) return st;
  return BA_OK;
}

ba_status ba_get_blocks(ba_handle* h, double* U, double* V, double* b_p, double* b_l, int32_t ptr_kind) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!h->linearized) return fail(BA_ERR_NOT_LINEARIZED, "no current linearisation");
  if (ptr_kind != 0 && ptr_kind != 1) return fail(BA_ERR_INVALID_ARG, "ptr_kind must be 0 or 1");
  CK(cudaStreamSynchronize(h->stream));
  const int nc = h->n_c, nl = h->n_l;
  ba_status st;
  if (U) {
    std::vector<double> u45((size_t)nc * 45), u((size_t)nc * 81);
    CK(cudaMemcpy(u45.data(), h->U45, sizeof(double) * u45.size(), cudaMemcpyDeviceToHost));
    for (int c = 0; c < nc; ++c) {
      int idx = 0;
      for (int i = 0; i < 9; ++i)
        for (int j = i; j < 9; ++j, ++idx) {
          u[(size_t)c * 81 + i * 9 + j] = u45[(size_t)c * 45 + idx];
          u[(size_t)c * 81 + j * 9 + i] = u45[(size_t)c * 45 + idx];
        }
    }
    if ((st = copy_out(U, u.data(), sizeof(double) * u.size(), ptr_kind)) != BA_OK) return st;
  }
  if (b_p) {
    std::vector<double> b((size_t)nc * 9);
    CK(cudaMemcpy(b.data(), h->b_p, sizeof(double) * b.size(), cudaMemcpyDeviceToHost));
    if ((st = copy_out(b_p, b.data(), sizeof(double) * b.size(), ptr_kind)) != BA_OK) return st;
  }
  if (V) {
    std::vector<double> v6((size_t)h->n_li * 6), v((size_t)nl * 9);
    CK(cudaMemcpy(v6.data(), h->V, sizeof(double) * v6.size(), cudaMemcpyDeviceToHost));
    static const int map[9] = {0, 1, 2, 1, 3, 4, 2, 4, 5};
    for (int i = 0; i < h->n_li; ++i) {
      const size_t c = (size_t)h->sched.lm_order[i];
      for (int k = 0; k < 9; ++k) v[c * 9 + k] = v6[(size_t)i * 6 + map[k]];
    }
    if ((st = copy_out(V, v.data(), sizeof(double) * v.size(), ptr_kind)) != BA_OK) return st;
  }
  if (b_l) {
    std::vector<double> bi((size_t)h->n_li * 3), bo((size_t)nl * 3);
    CK(cudaMemcpy(bi.data(), h->b_l, sizeof(double) * bi.size(), cudaMemcpyDeviceToHost));
    for (int i = 0; i < h->n_li; ++i)
      for (int k = 0; k < 3; ++k) bo[(size_t)h->sched.lm_order[i] * 3 + k] = bi[(size_t)i * 3 + k];
    if ((st = copy_out(b_l, bo.data(), sizeof(double) * bo.size(), ptr_kind)) != BA_OK) return st;
  }
  return BA_OK;
}

ba_status ba_get_lm_state(ba_handle* h, double* lambda, double* nu, int32_t* iteration, double* cost) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (h->n_probs != 1)
    return fail(BA_ERR_INVALID_ARG, "a batch handle reports its LM state per problem (ba_lm_step_batch)");
  CK(cudaMemcpyAsync(h->h_rec, h->rec, sizeof(LmRecord), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (lambda) *lambda = h->h_rec->lambda;
  if (nu) *nu = h->h_rec->nu;
  if (iteration) *iteration = h->h_rec->iteration;
  if (cost) *cost = h->cost_valid ? h->h_rec->cost : NAN;
  return BA_OK;
}

ba_status ba_set_lm_state(ba_handle* h, double lambda, double nu, int32_t iteration) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (!(lambda > 0.0) || !std::isfinite(lambda) || !(nu >= 1.0) || !std::isfinite(nu) || iteration < 0)
    return fail(BA_ERR_INVALID_ARG, "need lambda > 0, nu >= 1, iteration >= 0");
  const size_t P = (size_t)h->n_probs;
  CK(cudaMemcpyAsync(h->h_rec, h->rec, sizeof(LmRecord) * P, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t p = 0; p < P; ++p) {
    LmRecord& r = h->h_rec[p];
    r.lambda = lambda;
    r.nu = nu;
    r.iteration = iteration;
    r.converged = 0;
    r.active = 1;
  }
  CK(cudaMemcpyAsync(h->rec, h->h_rec, sizeof(LmRecord) * P, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return BA_OK;
}

ba_status ba_get_series_trace(ba_handle* h, int64_t* ns, int32_t capacity, int32_t* n_terms) {
  if (!h || !ns || capacity < 0) return fail(BA_ERR_INVALID_ARG, "bad argument");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->h_st, h->st, sizeof(SeriesState) * h->n_probs, cudaMemcpyDeviceToHost));
  int terms = h->last_exec >= 3 ? max_terms(h) : 0;
  if (terms > kTraceTerms) terms = kTraceTerms;
  const int n = terms * kTracePoints < capacity ? terms * kTracePoints : capacity;
  if (n > 0) CK(cudaMemcpy(ns, h->trace, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
  if (n_terms) *n_terms = terms;
  return BA_OK;
}

ba_status ba_set_barrier_timeout(ba_handle* h, int64_t cycles) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  h->barrier_timeout = cycles < 1 ? (1LL << 33) : (long long)cycles;
  return BA_OK;
}

ba_status ba_memory_footprint(ba_handle* h, uint64_t* bytes) {
  if (!h || !bytes) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  *bytes = (uint64_t)(h->arena_bytes + h->ser_bytes);
  return BA_OK;
}

ba_status ba_kernel_launches(ba_handle* h, uint64_t* count) {
  if (!h || !count) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  *count = h->launches;
  return BA_OK;
}

ba_status ba_set_timing(ba_handle* h, int32_t enable) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  CK(cudaStreamSynchronize(h->stream));
  h->timing = enable != 0;
  for (int c = 0; c < BA_TIMING_CLASSES; ++c) {
    h->t_ms[c] = 0.0;
    h->t_count[c] = 0;
    h->pending[c] = false;
  }
  if (h->timing) return ensure_events(h);
  return BA_OK;
}

ba_status ba_get_timing(ba_handle* h, ba_timing* out) {
  if (!h || !out) return fail(BA_ERR_INVALID_ARG, "NULL argument");
  for (int c = 0; c < BA_TIMING_CLASSES; ++c) {
    out->ms[c] = h->t_ms[c];
    out->count[c] = h->t_count[c];
  }
  return BA_OK;
}

ba_status ba_debug_checks(ba_handle* h, int32_t* enabled, uint32_t* site, uint32_t* count,
                          int64_t* index) {
  if (!h) return fail(BA_ERR_INVALID_ARG, "handle is NULL");
  if (enabled) *enabled = kChecks ? 1 : 0;
  if (site) *site = 0;
  if (count) *count = 0;
  if (index) *index = 0;
  if (!kChecks) return BA_OK;
  cudaStream_t s = h->stream;
  if (h->canary_n[0] > 0)
    launch_canary_check((const uint8_t*)h->arena, h->canary_dev[0], h->canary_n[0], kChkCanary,
                        h->chk, s);
  if (h->canary_n[1] > 0 && h->ser_arena)
    launch_canary_check((const uint8_t*)h->ser_arena, h->canary_dev[1], h->canary_n[1],
                        kChkCanary + 1000, h->chk, s);
  CheckRecord r{};
  CK(cudaMemcpyAsync(&r, h->chk, sizeof(r), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemsetAsync(h->chk, 0, sizeof(CheckRecord), s));
  if (site) *site = r.site;
  if (count) *count = r.count;
  if (index) *index = r.index;
  return BA_OK;
}

const char* ba_status_string(ba_status s) {
  switch (s) {
    case BA_OK: return "BA_OK";
    case BA_ERR_INVALID_ARG: return "BA_ERR_INVALID_ARG";
    case BA_ERR_CUDA: return "BA_ERR_CUDA";
    case BA_ERR_OOM: return "BA_ERR_OOM";
    case BA_ERR_NOT_SPD: return "BA_ERR_NOT_SPD";
    case BA_ERR_NONFINITE: return "BA_ERR_NONFINITE";
    case BA_ERR_NOT_LINEARIZED: return "BA_ERR_NOT_LINEARIZED";
    case BA_ERR_TIMEOUT: return "BA_ERR_TIMEOUT";
    case BA_ERR_CHECK: return "BA_ERR_CHECK";
  }
  return "unknown status";
}

const char* ba_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
