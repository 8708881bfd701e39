// Debug-build checks of libpoba (compiled with -DPOBA_CHECKS into libpoba_checks.so; a release
// build compiles every check away).
//
// Index checks: before a kernel uses an index read from the schedule (a camera or landmark of
// an observation, a slot, a position or a segment bound), POBA_CHK tests it against its bound.
// A failed test records the site, the index and the bound in the handle's CheckRecord (the
// first failure wins; later ones only count) and replaces the index by 0, so that the access
// stays in bounds and the kernel runs to its end (no trap: the context stays usable).  The host
// reads the record after each synchronising call and reports BA_ERR_CHECK.
//
// Canaries: every sub-buffer of the handle's device allocations is followed by kCanaryBytes
// bytes of kCanaryByte, checked by a kernel at the same points; a changed byte records site
// kChkCanary + the sub-buffer's index.
#pragma once

#include <cstdint>

namespace poba {

struct CheckRecord {
  unsigned site;     // first failed check (0: none)
  unsigned count;    // failed checks since the record was cleared
  long long index;   // the offending index of the first failure
  long long bound;   // its bound
};

enum CheckSite : unsigned {
  kChkNone = 0,
  kChkLinCam = 1,        // linearisation: camera of an observation
  kChkLinLm = 2,         // linearisation: landmark of an observation
  kChkLinPos = 3,        // linearisation: camera-sorted position of an observation
  kChkLinSlot = 4,       // linearisation: tile slot of an observation
  kChkLinSeg = 5,        // linearisation: slot segment bound
  kChkLinRow = 6,        // linearisation: camera-major row of a tile slot
  kChkCamReduce = 7,     // camera reduction: slot row range of a camera
  kChkCostCam = 8,       // cost: camera of an observation
  kChkCostLm = 9,        // cost: landmark of an observation
  kChkBackCam = 10,      // back-substitution: camera of a tile slot
  kChkBackSlot = 11,     // back-substitution: tile slot of an observation
  kChkBackSeg = 12,      // back-substitution: landmark segment of a tile
  kChkSerCam = 13,       // series: camera of a group slot
  kChkSerRow = 14,       // series: partial row of a group slot
  kChkChunkPos = 15,     // series: position in a chunk's camera-sorted order
  kChkChunkSlot = 16,    // series: group slot of an observation
  kChkChunkLm = 17,      // series: landmark of an observation within its chunk
  kChkChunkSeg = 18,     // series: landmark segment bound within a chunk
  kChkClistSlot = 19,    // series: group slot of a chunk slot
  kChkClistSeg = 20,     // series: row range of a chunk slot
  kChkCamRows = 21,      // camera step: partial-row range of a camera
  kChkLongSeg = 22,      // long track: observation range of a piece
  kChkCanary = 100,      // + the index of the sub-buffer whose guard bytes changed
};

constexpr int kCanaryBytes = 256;
constexpr unsigned char kCanaryByte = 0xA5;

#ifdef POBA_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif

#if defined(POBA_CHECKS) && defined(__CUDACC__)
__device__ __forceinline__ long long chk_index(CheckRecord* r, unsigned site, long long i,
                                               long long bound) {
  if (i >= 0 && i < bound) return i;
  if (r) {
    if (atomicCAS(&r->site, 0u, site) == 0u) {
      r->index = i;
      r->bound = bound;
    }
    atomicAdd(&r->count, 1u);
  }
  return 0;
}
// i must be an lvalue of an integer type; bound is exclusive
#define POBA_CHK(rec, i, bound, site) \
  ((i) = (decltype(i))::poba::chk_index((rec), (site), (long long)(i), (long long)(bound)))
#else
#define POBA_CHK(rec, i, bound, site) ((void)0)
#endif

}  // namespace poba
