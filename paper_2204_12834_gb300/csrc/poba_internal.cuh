// Internal declarations of libpoba: device data layout, kernel launchers, host schedule.
//
// Data layout in HBM (all per-handle, one arena allocation):
//   Observations are stored sorted by (internal landmark, camera).  Internal landmark order
//   groups landmarks by their smallest observing camera so that a run of consecutive
//   landmarks touches few cameras.  Consecutive landmarks are packed into tiles of at most
//   kTileObs observations; a landmark never straddles two tiles (its "memory block" in the
//   sense of Sec. 5, "Efficient storage").  Per tile, the distinct cameras form "slots"; the
//   camera-keyed reductions (W y scatter and J_p^T J_p) sum per slot inside the tile and then
//   per camera across the slots that camera owns (CSR cam_slot_ptr / cam_slot_list), so no
//   global atomics are used and every sum has a fixed order.
//
//   Per-slot partial sums are written camera-major (row slot_row[s] of slot s), so the rows of
//   one camera are contiguous for the camera-side kernels.  A camera's rows are summed in
//   chunks of cam_chunk_rows(rows) rows (each chunk in row order, then the chunks in order), in
//   every kernel, so that the persistent kernels can spread a camera's chunks over threads and
//   still produce the same sums.  The current series term is kept per camera (t_cam, rows of
//   kTStride elements), which a tile gathers through its slots' cameras.  A tile holds at most
//   kTileSlots slots.
//
//   Jacobians are 24 planes p (p = 0..17: J_p row-major, row i, col j at p = 9 i + j;
//   p = 18..23: J_l row-major at p = 18 + 3 i + j) in the handle's bulk precision T, stored in
//   16-byte plane groups: the V = 16 / sizeof(T) planes V q .. V q + V - 1 of observation o are
//   contiguous at J[(q * n_obs_pad + o) * V] (jidx below), so a thread reads its observation's 24
//   values with 6 (float) or 12 (double) 16-byte loads, and one load instruction of a warp covers
//   512 contiguous bytes.  Residuals are planes of length n_obs_pad: r[i * n_obs_pad + o].
//   obs_meta[o] (uint16) = (position of o in the tile's camera-sorted order) | slot << 8.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "checks.cuh"

namespace poba {

constexpr int kTileObs = 256;   // observations per tile (= threads of the tile kernels)
constexpr int kTileLms = 256;   // landmarks per tile
constexpr int kTileSlots = 128; // distinct cameras (slots) per tile
constexpr int kTStride = 12;    // elements per camera row of the current term (9 used; 16-byte
                                // aligned rows for asynchronous copies)
constexpr int kCamChunkMin = 64;  // rows per chunk of a camera's row sum (at least): few
                                  // rounds for cameras with many slot rows
constexpr int kRoundItems = 28;   // camera chunks per round of the persistent camera phase

// Rows per chunk of a camera with `rows` slot rows: at least kCamChunkMin, and few enough
// chunks to fit one round.
__host__ __device__ constexpr int cam_chunk_rows(int rows) {
  return (rows + kRoundItems - 1) / kRoundItems > kCamChunkMin
             ? (rows + kRoundItems - 1) / kRoundItems
             : kCamChunkMin;
}
__host__ __device__ constexpr int cam_chunks(int rows) {
  return rows > 0 ? (rows + cam_chunk_rows(rows) - 1) / cam_chunk_rows(rows) : 1;
}
constexpr int kLinVals = 54;    // 45 packed upper-triangular entries of J_p^T J_p + 9 of J_p^T r
constexpr int kCamBlock = 32;   // cameras per block in the damp / invert kernel
constexpr int kReduceThreads = 256;

// ---------------------------------------------------------------------------------------
// Host-side tile schedule (built once in ba_create).
struct Schedule {
  int n_cams = 0, n_lms = 0, n_obs = 0, n_probs = 1;
  int n_tiles = 0, n_slots = 0, max_slots_per_tile = 0, max_track = 0;
  // Internal landmarks: a landmark with more than kTileObs observations (a long track) is
  // split into near-equal pieces of at most kTileObs observations in camera order, each an
  // internal landmark with its own tile and a copy of the landmark's state; its landmark-side
  // sums are combined over the pieces in piece order.  n_lms_int counts internal landmarks.
  int n_lms_int = 0, n_long = 0;
  std::vector<int32_t> long_first;   // [n_long] first piece (internal landmark) of each long track
  std::vector<int32_t> long_np;      // [n_long] its pieces
  std::vector<int32_t> long_tile0;   // [n_long] the tile of its first piece (one tile per piece)
  std::vector<int32_t> lm_long;      // [n_lms_int] long track of each internal landmark, or -1
  std::vector<int32_t> lm_order;     // internal landmark -> caller landmark
  std::vector<int32_t> lm_rank;      // caller landmark -> (first) internal landmark
  std::vector<int64_t> obs_order;    // sorted observation -> caller observation
  std::vector<int32_t> lm_seg;       // [n_lms_int + 1] observation offsets per internal landmark
  std::vector<int32_t> cam_of;       // [n_obs] camera of each sorted observation
  std::vector<int32_t> lm_of;        // [n_obs] internal landmark of each sorted observation
  std::vector<uint16_t> obs_meta;    // [n_obs] pos | slot << 8
  std::vector<int32_t> tile_lm0;     // [n_tiles + 1]
  std::vector<int32_t> tile_slot0;   // [n_tiles + 1]
  std::vector<int32_t> tile_desc;    // [n_tiles][8]: L0, n_lms, o0, n_obs, S0, n_slots, rec, prob
  std::vector<uint8_t> tile_rec;     // per-tile records (see tile_rec_layout), 16-byte aligned
  std::vector<int32_t> slot_cam;     // [n_slots]
  std::vector<uint16_t> slot_beg;    // [n_slots] first camera-sorted position of the slot
  std::vector<int32_t> cam_slot_ptr; // [n_cams + 1]
  std::vector<int32_t> cam_slot_list;// [n_slots] camera-major row -> tile-major slot
  std::vector<int32_t> slot_row;     // [n_slots] tile-major slot -> camera-major row
  // independent problems (a batch): cameras [cam_off[p], cam_off[p+1]) and caller landmarks
  // [lm_off[p], lm_off[p+1]) form problem p; internal landmarks and tiles are contiguous per
  // problem and no tile holds two problems
  std::vector<int32_t> cam_off;      // [n_probs + 1]
  std::vector<int32_t> lm_off_int;   // [n_probs + 1] internal landmark ranges
  std::vector<int32_t> tile_off;     // [n_probs + 1] tile ranges
  std::vector<int32_t> cam_prob;     // [n_cams]
  std::vector<int32_t> lm_prob;      // [n_lms_int] problem of each internal landmark
};

// Per-tile record, one contiguous 16-byte aligned block per tile, so that one bulk copy brings
// a tile's index data into shared memory: the observations' codes (pos | slot << 8), their
// landmark within the tile, the slots' first positions, the landmark segment offsets (tile-
// relative), the slots' camera-major rows and the slots' cameras.  Each array is padded to a multiple of 16 bytes.
// tile_desc[t][6] is the record's offset in 16-byte units.
struct TileRecLayout {
  int meta, olm, sbeg, sseg, srow, scam, bytes;  // byte offsets of the arrays and the total
};
__host__ __device__ constexpr TileRecLayout tile_rec_layout(int n, int ns, int nl) {
  const int n8 = (n + 7) & ~7, n16 = (n + 15) & ~15, ns8 = (ns + 7) & ~7;
  const int nl8 = (nl + 1 + 7) & ~7, ns4 = (ns + 3) & ~3;
  const int meta = 0, olm = meta + 2 * n8, sbeg = olm + n16, sseg = sbeg + 2 * ns8;
  const int srow = sseg + 2 * nl8, scam = srow + 4 * ns4, bytes = scam + 4 * ns4;
  return TileRecLayout{meta, olm, sbeg, sseg, srow, scam, bytes};
}
constexpr int kTileRecMax = tile_rec_layout(kTileObs, kTileSlots, kTileLms).bytes;

// Jacobian plane groups (see the layout note above): elements of T per 16-byte group and the
// index of plane p of observation o.
template <typename T>
__host__ __device__ constexpr int jgroup() { return (int)(16 / sizeof(T)); }
template <typename T>
__host__ __device__ __forceinline__ size_t jidx(int p, size_t o, size_t pad) {
  return ((size_t)(p / jgroup<T>()) * pad + o) * jgroup<T>() + (size_t)(p % jgroup<T>());
}

// Returns an empty string on success, else a description of why the inputs are rejected.
// cam_off / lm_off ([n_probs + 1]) split cameras and landmarks into independent problems; every
// observation must join a camera and a landmark of the same problem.  NULL means one problem.
std::string build_schedule(int n_cams, int n_lms, int n_obs, const int32_t* cam_idx,
                           const int32_t* lm_idx, int n_probs, const int32_t* cam_off,
                           const int32_t* lm_off, Schedule* out);

// ---------------------------------------------------------------------------------------
// Series schedule (host, rebuilt when the group size changes).  The power-series kernels do
// not use the tiles above: each problem's observed landmarks are cut into groups of
// consecutive landmarks holding about `target` observations (boundaries at whole landmarks,
// balanced by observation count; a group also ends before it would touch more than
// kGroupSlots (FP64: kGroupSlotsF64) distinct cameras; optionally each group's last eighth is
// cut into smaller groups), and each group into chunks of at most kChunkObs observations of
// whole landmarks.  One block runs one group: its chunks in order, with one accumulator row
// per distinct camera of the group (a group slot), written once per group as a partial row.
// A camera's partial rows (one per group that touches it) are contiguous, groups in landmark
// order (cam_ptr), and summed by the camera kernels in chunks of cam_chunk_rows rows.
//
// Chunk record (16-byte aligned, chunk_rec_layout):
//   code[n]      uint32 per observation: position in the chunk's camera-sorted order (bits
//                0-7) | group slot of its camera (8-15) | landmark within the chunk (16-23);
//   sseg[nl + 1] uint16 landmark offsets within the chunk;
//   clist[ns]    uint32 per distinct camera of the chunk (a chunk slot): its group slot
//                (bits 0-7) | its first camera-sorted position (8-15) | its number of rows
//                (16-24); longest first (ties in camera order), so that the lanes that sum
//                one warp's slots have similar work.
constexpr int kChunkObs = 256;
constexpr int kGroupSlots = 256;     // distinct cameras of an FP32-bulk group (at most)
constexpr int kGroupSlotsF64 = 96;   // of an FP64 group, whose shared memory also holds a
                                     // chunk's J_p rows (the FP64 slot sums form J_p^T w)

struct ChunkRecLayout {
  int code, sseg, clist, bytes;
};
__host__ __device__ constexpr ChunkRecLayout chunk_rec_layout(int n, int nl, int ns) {
  return ChunkRecLayout{0, 4 * ((n + 3) & ~3), 4 * ((n + 3) & ~3) + 2 * ((nl + 1 + 7) & ~7),
                        4 * ((n + 3) & ~3) + 2 * ((nl + 1 + 7) & ~7) + 4 * ((ns + 3) & ~3)};
}
constexpr int kChunkRecMax = chunk_rec_layout(kChunkObs, kChunkObs, kChunkObs).bytes;

struct SerSchedule {
  int target = 0;  // observations per group the partition aimed at
  int tail = 0;    // pieces the last eighth of each group is cut into (0: none)
  int n_groups = 0, n_chunks = 0, n_gslots = 0, max_group_slots = 0;
  int n_long_groups = 0;  // groups run by the long-group body (long tracks, wide landmarks)
  // [n_groups][8] in ticket order (decreasing observation count): chunk0, n_chunks, gslot0,
  // n_gslots, n_obs, problem, 0, 0
  std::vector<int32_t> group;
  // [n_chunks][8] (landmark order): o0, n, L0, nl, ns, record offset / 16, group, 0
  std::vector<int32_t> chunk;
  std::vector<uint8_t> rec;         // chunk records
  std::vector<int32_t> gslot_cam;   // [n_gslots] camera of each group slot
  std::vector<int32_t> gslot_row;   // [n_gslots] its camera-major partial row
  std::vector<int32_t> cam_ptr;     // [n_cams + 1] partial rows of each camera
  std::vector<int32_t> prob_ncam;   // [n_probs] cameras of each problem with a partial row
};

// Builds the series schedule of S for a target group size (observations, >= 1).  tail > 0: the
// last eighth of the observations of each group (of at least two chunks) becomes `tail`
// smaller groups, which the ticket order (largest first) hands out last, so that blocks that
// finish their large group early take them and the phase ends more evenly.
std::string build_series_schedule(const Schedule& S, int target, int tail, SerSchedule* out,
                                  int slot_cap = kGroupSlots);
// The automatic group size for G blocks that run groups: one group of n_obs / G observations
// per block (at least one chunk's worth).
int series_auto_target(int64_t n_obs, int G);

// Camera schedule of the persistent camera phase.  Items are the chunks of every camera's slot
// rows (cam_chunks per camera, in camera order): camera c owns items [cam_item[c],
// cam_item[c + 1]) and item i covers rows [item_q[2 i], item_q[2 i + 1]).  Rounds pack whole
// cameras in order with at most max_items items (at most kRoundItems, at least the largest
// camera's chunk count): round r holds cameras [round_cam[r], round_cam[r + 1]) and items
// [round_item[r], round_item[r + 1]).  For a grid of G blocks, block b runs rounds
// [block_round[b], block_round[b + 1]).
struct CamSchedule {
  std::vector<int32_t> cam_item, item_q;
};
struct CamRoundList {
  std::vector<int32_t> round_cam, round_item, block_round;
};
void build_cam_schedule(const std::vector<int32_t>& cam_ptr, int n_cams, CamSchedule* out);
// Rounds sized for a grid of G blocks: as few items per round as spread the items over the grid.
void build_cam_rounds(const CamSchedule& cs, int n_cams, int G, CamRoundList* out);

struct CamRounds {
  const int32_t* cam_item;
  const int32_t* item_q;
  const int32_t* round_cam;
  const int32_t* round_item;
  const int32_t* block_round;  // [G + 1]
};

// ---------------------------------------------------------------------------------------
// Device views passed to kernels by value.
struct Topology {
  int n_cams, n_lms, n_obs, n_obs_pad, n_tiles, n_slots;
  const int32_t* lm_seg;
  const int32_t* cam_of;
  const int32_t* lm_of;
  const uint16_t* obs_meta;
  const int32_t* tile_lm0;
  const int32_t* tile_slot0;
  const int4* tile_desc;  // two int4 per tile: {L0, nl, o0, n}, {S0, ns, rec16, problem}
  const uint8_t* tile_rec;  // per-tile records (tile_rec_layout)
  const int32_t* slot_cam;
  const uint16_t* slot_beg;
  const int32_t* cam_slot_ptr;
  const int32_t* cam_slot_list;
  const int32_t* slot_row;  // partial sums are stored camera-major: row slot_row[slot]
  // long tracks (Schedule): their pieces, the tile of the first piece, the track of each
  // internal landmark (-1: none)
  int n_long;
  const int32_t* long_first;
  const int32_t* long_np;
  const int32_t* long_tile0;
  const int32_t* lm_long;
  CheckRecord* chk;  // debug-build index checks (checks.cuh)
  // independent problems (P = 1 for a single problem)
  int n_probs;
  const int32_t* cam_prob;  // [n_cams]
  const int32_t* lm_prob;   // [n_lms] (internal landmark order)
  const int32_t* tile_prob; // [n_tiles]
  const int32_t* cam_off;   // [n_probs + 1]
  const int32_t* tile_off;  // [n_probs + 1]
};

// Device view of the series schedule (SerSchedule), passed to the series kernels by value.
struct SerTopo {
  int n_groups, n_chunks, n_gslots;
  const int4* group;         // [n_groups][2]: {chunk0, n_chunks, gslot0, n_gslots}, {n_obs, problem, 0, 0}
  const int4* chunk;         // [n_chunks][2]: {o0, n, L0, nl}, {ns, record offset / 16, group, 0}
  const uint8_t* rec;        // chunk records (chunk_rec_layout)
  const int32_t* gslot_cam;  // [n_gslots]
  const int32_t* gslot_row;  // [n_gslots] camera-major partial row
  const int32_t* cam_ptr;    // [n_cams + 1] partial rows of each camera
  const int32_t* prob_ncam;  // [n_probs] cameras of each problem with at least one partial row
  int prefetch;              // 1: group bodies prefetch their next chunk to L2
};

// Per-launch state of the dataflow series kernel (series_exec 5), zeroed before each launch.
struct FlowState {
  unsigned* cam_cnt;   // [n_cams] group slots of camera c completed in this launch (all terms)
  int* cam_epoch;      // [n_cams] last term whose update of camera c is published
  unsigned* pcnt;      // [n_probs][2] camera updates completed, by term parity
  int* prob_dec;       // [n_probs] last term whose stop rule has been applied
  double* cam_norm_b;  // [n_cams][2] norm pairs of odd terms (even terms use cam_norm)
};
constexpr size_t flow_state_bytes(int n_cams, int n_probs) {
  return (size_t)n_cams * (4 + 4 + 16) + (size_t)n_probs * (8 + 4) + 64;
}

// Per-camera values prepared once per state: rotation R (row-major), the matrix G with
// dP/dw = -[Y]x G (Y = R X and G = left Jacobian of SO(3) on the regular branch; Y = X and
// G = I on the first-order branch), translation, intrinsics, and the branch flag.
constexpr int kCamPrep = 25;  // R[9] G[9] t[3] f k1 k2 first_order

// Series state (device), one per problem.
struct SeriesState {
  int32_t done;        // stop rule fired, or the problem takes no part in this solve
  int32_t m;           // number of P applications performed
  int32_t stopped;     // 1 if the stop test fired
  int32_t pad0;
  double stop_value;
  double x_norm;
  double t_norm;
  double pad1;
};

// Series state shared by all problems of a handle.
struct SeriesGlobal {
  int32_t all_done;    // every problem has stopped (later terms return at once)
  uint32_t counter;    // last-block ticket of the per-term camera kernel
  int32_t n_list;      // tiles in the active tile list (batches)
  int32_t n_running;   // problems still running after the last stop-rule pass
};

// Grid-barrier state of the persistent series kernel (zeroed before each launch).
struct GridSync {
  unsigned arrive;     // grid-barrier arrivals since the launch (barrier n completes at (n+1) G)
  int error;           // 1: a barrier wait timed out or a block failed
  unsigned pad0[30];   // the tile counter lives on its own 128-byte line
  unsigned tile_next;  // dynamic tile counter of the current tile phase
  unsigned pad1[31];
};

// LM record (device), written by the decide kernel and read by the host once per iteration.
struct LmRecord {
  double cost;          // F(x) (current state)
  double cost_before;   // F(x) before the last step
  double cost_trial;    // F(x + dx)
  double model_decrease;
  double gain_ratio;
  double lambda;        // damping for the next solve
  double nu;
  double lambda_used;
  int32_t accepted;
  int32_t not_spd;      // the last iteration's damped blocks were not positive definite
  int32_t nonfinite;
  int32_t iteration;
  int32_t converged;
  int32_t active;       // 0: the problem has converged and is frozen (batches only)
};

// Sets the thread's ba_last_error() message (defined with the C ABI).
void set_last_error(const std::string& msg);

// ---------------------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).  All take the stream last.
// prep32 (optional): a float copy of the records for the FP32-bulk linearisation.
// gate (optional, device): the kernels return at once when *gate == 0 (a captured LM step skips
// the linearisation when the last step was rejected; the flag is set on the device).
void launch_cam_prepare(const double* cams, const double* dx_p, int n_cams, double* prep,
                        double* cams_out, cudaStream_t s, float* prep32 = nullptr,
                        const int32_t* gate = nullptr);

// Pair type of the observations in a precision: double2 / float2.
template <typename T> struct Vec2Of;
template <> struct Vec2Of<double> { using type = double2; };
template <> struct Vec2Of<float> { using type = float2; };
template <typename T> using vec2 = typename Vec2Of<T>::type;

// Inputs in the working precision T: the prepared camera records, the observations and the
// square-root weights (FP32 bulk passes float copies made once, so that no observation pays a
// double-to-float conversion, which GB300 runs on its FP64 pipe).
template <typename T>
void launch_linearize(const Topology& tp, const T* prep, const double* lms, const vec2<T>* obs,
                      const T* sqrt_w, T* J, T* r, double* V, double* b_l, T* partial,
                      double* block_cost, cudaStream_t s, const int32_t* gate = nullptr);

template <typename PT>
void launch_lin_camera_reduce(const Topology& tp, const PT* partial, double* U45, double* b_p,
                              cudaStream_t s, const int32_t* gate = nullptr);

// lambda of problem p is lam[p * lam_stride] (lam_stride 0: one lambda for all problems);
// not_spd[p] is set to 1 when a damped block of problem p fails its Cholesky factorisation (the
// failed pivot is replaced by 1 so that the inverse stays finite).
// Debug builds: guard bytes of an allocation (checks.cuh).
void launch_canary_check(const uint8_t* base, const uint64_t* off, int n, unsigned site0,
                         CheckRecord* chk, cudaStream_t s);
// Long tracks: V and b_l summed over each track's pieces and written back to every piece.
void launch_long_track_blocks(const Topology& tp, double* V, double* b_l, cudaStream_t s,
                              const int32_t* gate = nullptr);
void launch_damp_invert(const Topology& tp, const double* U45, const double* V,
                        const double* lambda, int lam_stride, int damping_mode, double* Uinv,
                        double* Vinv, float* Vinv_f, int32_t* not_spd, cudaStream_t s);

// 2 F per tile (sum of w ||r||^2 over the tile's observations) at (cameras in prep, landmarks
// lms + dx_l), float64.
void launch_tile_cost(const Topology& tp, const double* prep, const double* lms,
                      const double* dx_l, const double2* obs, const double* sqrt_w,
                      double* tile_cost, cudaStream_t s);

// Series kernels over the series schedule sp (one block per group): b~'s tile part
// W V^-1 b_l (RHS) or W V^-1 W^T t (series) as partial rows, then the camera kernels.
// series_group_kernels_init raises the kernels' dynamic shared-memory limit (once per process).
template <typename T>
cudaError_t series_group_kernels_init();

template <typename T>
void launch_tile_rhs(const Topology& tp, const SerTopo& sp, const T* J, const double* b_l,
                     const T* Vinv, T* partial, const SeriesState* st, cudaStream_t s);

template <typename T>
void launch_tile_series(const Topology& tp, const SerTopo& sp, const T* J, const T* t_cam,
                        const T* Vinv, T* partial, const SeriesState* st, const SeriesGlobal* sgl,
                        cudaStream_t s);

template <typename T>
void launch_tile_backsub(const Topology& tp, const T* J, const T* r, const double* x,
                         const double* b_l, const T* Vinv, double* dx_l,
                         double* block_pred, cudaStream_t s);

// The camera kernels sum each camera's partial rows (sp.cam_ptr), write the new term t into the
// camera's row of t_cam, which the next group kernel gathers, and a (||t_c||^2, ||x_c||^2) pair
// per camera (cam_norm); the last block to finish reduces the pairs per problem and applies the
// stop rule of each problem.
template <typename PT>
void launch_camera_rhs(const Topology& tp, const SerTopo& sp, const PT* partial, const double* b_p,
                       const double* Uinv, double* x, PT* t_cam, double* cam_norm,
                       SeriesState* st, SeriesGlobal* sgl, cudaStream_t s);

template <typename PT>
void launch_camera_series(const Topology& tp, const SerTopo& sp, const PT* partial,
                          const double* Uinv, double* x, PT* t_cam, double* cam_norm,
                          SeriesState* st, SeriesGlobal* sgl, int iter, double eps,
                          cudaStream_t s);

int camera_blocks(const Topology& tp);

// done[p] = 1 for problems that take no part (rec[p].active == 0; rec may be NULL).
void launch_series_reset(SeriesState* st, SeriesGlobal* sgl, const LmRecord* rec, int n_probs,
                         cudaStream_t s);

// out[p * out_stride] = scale * (sum of tile_vals over the tiles of problem p), fixed order.
void launch_reduce_tiles(const Topology& tp, const double* tile_vals, double* out,
                         int out_stride, double scale, cudaStream_t s);

// Per problem: F(x + dx) and the model decrease from tile sums, gain ratio, accept, lambda / nu
// update; inactive problems are left as they are.  A problem whose damped blocks were not
// positive definite (not_spd[p]) has no step: it is rejected.  deactivate: a converged problem
// becomes inactive.
// relin (optional, device): set to 1 when any problem's step was accepted (the state moved,
// so the next step linearises).
void launch_lm_decide(const Topology& tp, const double* tile_cost, const double* tile_pred,
                      const int32_t* not_spd, LmRecord* rec, double func_tol, int deactivate,
                      cudaStream_t s, int32_t* relin = nullptr);

void launch_apply_step(const Topology& tp, const LmRecord* rec, double* cams,
                       const double* cams_trial, double* lms, const double* dx_l,
                       cudaStream_t s);

void launch_set_scalar(double* dst, double v, cudaStream_t s);

// State input / output: *bad |= 1 if any of src[0..n) is not finite; dst[i] (internal order)
// = src[order[i]] (rows of 3); dst[order[i]] = src[i].
void launch_check_finite(const double* src, int n, int32_t* bad, cudaStream_t s);
void launch_gather_rows3(const double* src, const int32_t* order, int n, double* dst, cudaStream_t s);
void launch_scatter_rows3(const double* src, const int32_t* order, int n, double* dst, cudaStream_t s);

// PCG on the reduced camera system (kernels_pcg.cu).  Scalars of the recursion, in sc[]:
enum { kPcgRz = 0, kPcgPq = 1, kPcgRzNew = 2, kPcgRr = 3, kPcgBb = 4, kPcgZero = 5, kPcgCount = 8 };
constexpr int kPcgDotBlocks = 128;
template <typename T>
void launch_schur_jacobi_tiles(const Topology& tp, const T* J, const double* Vinv, T* partial,
                               cudaStream_t s);
void launch_schur_diag(int n_cams, const double* U45, const double* SJ45, double lam, int mode,
                       double* S45, cudaStream_t s);
void launch_invert_camera_blocks(const Topology& tp, const double* A45, const double* lambda,
                                 int damping_mode, double* out81, int32_t* not_spd,
                                 cudaStream_t s);
template <typename PT>
void launch_schur_camera(const Topology& tp, const SerTopo& sp, const PT* partial,
                         const double* U45, double lam, int mode, const double* p, double* q,
                         cudaStream_t s);
template <typename PT>
void launch_schur_rhs_camera(const Topology& tp, const SerTopo& sp, const PT* partial,
                             const double* b_p, double* out, cudaStream_t s);
template <typename PT>
void launch_stage_term(int n_cams, const double* p, PT* t_cam, cudaStream_t s);
void launch_dot(int n, const double* a, const double* b, double* part, double* out,
                cudaStream_t s);
void launch_cg_update(int n, const double* sc, const double* p, const double* q, double* y,
                      double* r, cudaStream_t s);
void launch_cg_direction(int n, double* sc, const double* z, double* p, int first,
                         cudaStream_t s);
void launch_block_apply(int n_cams, const double* M81, const double* r, double* z,
                        cudaStream_t s);
void launch_negate(int n, const double* src, double* dst, cudaStream_t s);

// Adjoint (kernels_adjoint.cu): the right-hand side -(dL/dx) in internal order, and the
// per-observation gradients dL/dobs (d_obs [n_obs][2]) and dL/dw (d_w [n_obs], may be NULL) in
// the caller's observation order from the adjoint vector (a_p per camera, a_l per internal
// landmark).
void launch_adjoint_rhs(int n_cams, int n_lms, const int32_t* lm_order, const double* g_p,
                        const double* g_l, double* adj_p, double* adj_l, cudaStream_t s);
template <typename T>
void launch_obs_gradient(const Topology& tp, const T* J, const T* r, const double* sqrt_w,
                         const double* a_p, const double* a_l, const int32_t* obs_caller,
                         double* d_obs, double* d_w, cudaStream_t s);

// Fixed-order sum of n doubles into *out = scale * sum (one block).
void launch_reduce_sum(const double* in, int n, double* out, double scale, cudaStream_t s);

// Persistent series kernel (cooperative launch): up to m_max terms and the stop rule.  Blocks
// take groups of the series schedule by ticket (sp.group is in ticket order), except the
// grid's last block, which applies the stop rule.  Block 0 records %globaltimer at 5 points of
// each of the first kTraceTerms terms (start, end of its group phase, after the first barrier,
// end of the camera phase, after the second barrier).
constexpr int kTraceTerms = 64;
constexpr int kTracePoints = 5;
int persistent_blocks_per_sm(bool f32);  // 0: the kernel cannot be launched on this device
// FP32-bulk persistent kernel with chunks staged in shared memory by bulk copies issued one
// chunk ahead (series_exec 4); the same sums as every other form.
int staged_blocks_per_sm();  // 0: the kernel cannot be launched on this device
cudaError_t launch_series_staged(const Topology& tp, const SerTopo& sp, const CamRounds& cr,
                                 int grid, const float* J, const float* Vinv, const double* Uinv,
                                 double* x, float* t_cam, float* partial, double* cam_norm,
                                 SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                 double eps, long long timeout, long long* trace,
                                 cudaStream_t s);
// Dataflow persistent kernel (series_exec 5): no grid barriers; per-camera counters and
// published term numbers order the work (see kernels_persistent.cu).
template <typename T>
int dataflow_blocks_per_sm();  // 0: the kernel cannot be launched on this device
template <typename T>
cudaError_t launch_series_dataflow(const Topology& tp, const SerTopo& sp, const FlowState& fs,
                                   int grid, const T* J, const T* Vinv, const double* Uinv,
                                   double* x, T* t_cam, T* partial, double* cam_norm,
                                   SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                   double eps, long long timeout, long long* trace,
                                   cudaStream_t s);
template <typename T>
cudaError_t launch_series_persistent(const Topology& tp, const SerTopo& sp, const CamRounds& cr,
                                     int grid, const T* J, const T* Vinv, const double* Uinv,
                                     double* x, T* t_cam, T* partial, double* cam_norm,
                                     SeriesState* st, SeriesGlobal* sgl, GridSync* gs, int m_max,
                                     double eps, long long timeout, long long* trace,
                                     cudaStream_t s);

}  // namespace poba
