// Host-side tile schedule for libpoba (built once per problem in ba_create).
//
// Sec. 5 ("Efficient storage") groups the Jacobians and residuals of each landmark into one
// dense memory block.  The GPU layout keeps that grouping and adds what the camera-keyed
// reductions need on a GPU: landmarks are ordered by their smallest observing camera, packed
// into tiles of at most kTileObs observations, and each tile's distinct cameras become slots
// whose sums are later combined per camera in a fixed order.
#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>
#include <string>

#include "poba_internal.cuh"

namespace poba {

std::string build_schedule(int n_cams, int n_lms, int n_obs, const int32_t* cam_idx,
                           const int32_t* lm_idx, int n_probs, const int32_t* cam_off,
                           const int32_t* lm_off, Schedule* S) {
  if (n_cams < 1 || n_lms < 1 || n_obs < 0) return "n_cams and n_lms must be >= 1, n_obs >= 0";
  if (n_probs < 1) return "need at least one problem";
  S->n_cams = n_cams;
  S->n_lms = n_lms;
  S->n_obs = n_obs;
  S->n_probs = n_probs;
  S->cam_off.assign(n_probs + 1, 0);
  std::vector<int32_t> loff(n_probs + 1, 0);
  if (cam_off && lm_off) {
    for (int p = 0; p <= n_probs; ++p) {
      S->cam_off[p] = cam_off[p];
      loff[p] = lm_off[p];
    }
  } else {
    if (n_probs != 1) return "problem offsets missing";
    S->cam_off[1] = n_cams;
    loff[1] = n_lms;
  }
  if (S->cam_off[0] != 0 || S->cam_off[n_probs] != n_cams || loff[0] != 0 || loff[n_probs] != n_lms)
    return "problem offsets must start at 0 and end at n_cams / n_lms";
  for (int p = 0; p < n_probs; ++p)
    if (S->cam_off[p + 1] <= S->cam_off[p] || loff[p + 1] <= loff[p])
      return "every problem needs at least one camera and one landmark";
  S->cam_prob.assign(n_cams, 0);
  for (int p = 0; p < n_probs; ++p)
    for (int c = S->cam_off[p]; c < S->cam_off[p + 1]; ++c) S->cam_prob[c] = p;
  std::vector<int32_t> lprob(n_lms, 0);
  for (int p = 0; p < n_probs; ++p)
    for (int l = loff[p]; l < loff[p + 1]; ++l) lprob[l] = p;

  std::vector<int32_t> count(n_lms, 0);
  std::vector<int32_t> key(n_lms, n_cams);  // smallest observing camera (n_cams if unobserved)
  for (int o = 0; o < n_obs; ++o) {
    int c = cam_idx[o], l = lm_idx[o];
    if (c < 0 || c >= n_cams) return "cam_idx[" + std::to_string(o) + "] out of range";
    if (l < 0 || l >= n_lms) return "lm_idx[" + std::to_string(o) + "] out of range";
    if (S->cam_prob[c] != lprob[l])
      return "observation " + std::to_string(o) + " joins a camera and a landmark of different problems";
    count[l]++;
    key[l] = std::min(key[l], c);
  }
  int max_track = 0;
  for (int l = 0; l < n_lms; ++l) max_track = std::max(max_track, count[l]);
  S->max_track = max_track;

  // Landmark order: by problem, then smallest observing camera (unobserved landmarks last
  // within their problem), then caller index.
  std::vector<int32_t> order(n_lms);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (lprob[a] != lprob[b]) return lprob[a] < lprob[b];
    return key[a] < key[b];
  });
  // Internal landmarks: the landmarks in that order, a long track as its pieces.
  std::vector<int32_t> first(n_lms);  // first internal landmark of each caller landmark
  int n_int = 0;
  S->long_first.clear();
  S->long_np.clear();
  for (int i = 0; i < n_lms; ++i) {
    const int l = order[i], k = count[l];
    first[l] = n_int;
    const int np = k > kTileObs ? (k + kTileObs - 1) / kTileObs : 1;
    if (np > 1) {
      S->long_first.push_back(n_int);
      S->long_np.push_back(np);
    }
    n_int += np;
  }
  S->n_lms_int = n_int;
  S->n_long = (int)S->long_first.size();
  S->lm_order.resize(n_int);
  S->lm_prob.resize(n_int);
  S->lm_long.assign(n_int, -1);
  S->lm_seg.assign(n_int + 1, 0);
  S->lm_off_int.assign(n_probs + 1, 0);
  for (int i = 0, j = 0; i < n_lms; ++i) {
    const int l = order[i], k = count[l];
    const int np = k > kTileObs ? (k + kTileObs - 1) / kTileObs : 1;
    for (int q = 0; q < np; ++q) {
      const int e = first[l] + q;
      S->lm_order[e] = l;
      S->lm_prob[e] = lprob[l];
      // piece q of np: near-equal sizes, the larger ones first
      S->lm_seg[e + 1] = S->lm_seg[e] + k / np + (q < k % np ? 1 : 0);
      S->lm_off_int[lprob[l] + 1]++;
    }
    if (np > 1) {
      for (int q = 0; q < np; ++q) S->lm_long[first[l] + q] = j;
      ++j;
    }
  }
  for (int p = 0; p < n_probs; ++p) S->lm_off_int[p + 1] += S->lm_off_int[p];
  S->lm_rank.assign(n_lms, 0);
  for (int l = 0; l < n_lms; ++l) S->lm_rank[l] = first[l];

  // Observations sorted by (landmark in internal order, camera, caller index); a long track's
  // observations go to its pieces in that order.
  S->obs_order.resize(n_obs);
  std::iota(S->obs_order.begin(), S->obs_order.end(), (int64_t)0);
  std::sort(S->obs_order.begin(), S->obs_order.end(), [&](int64_t a, int64_t b) {
    int la = S->lm_rank[lm_idx[a]], lb = S->lm_rank[lm_idx[b]];
    if (la != lb) return la < lb;
    if (cam_idx[a] != cam_idx[b]) return cam_idx[a] < cam_idx[b];
    return a < b;
  });
  S->cam_of.resize(n_obs);
  S->lm_of.resize(n_obs);
  for (int e = 0; e < n_int; ++e)
    for (int o = S->lm_seg[e]; o < S->lm_seg[e + 1]; ++o) {
      S->cam_of[o] = cam_idx[S->obs_order[o]];
      S->lm_of[o] = e;
    }

  // Tiles: greedy packing of whole landmarks of one problem, at most kTileObs observations,
  // kTileLms landmarks and kTileSlots distinct cameras per tile.
  S->tile_lm0.clear();
  S->tile_lm0.push_back(0);
  {
    int tile_obs = 0, tile_lms = 0, tile_cams = 0, tile_id = 0;
    std::vector<int32_t> stamp(n_cams, -1);  // tile that last counted the camera
    for (int i = 0; i < n_int; ++i) {
      const int k = S->lm_seg[i + 1] - S->lm_seg[i];
      int fresh = 0;  // cameras of landmark i not yet in the tile (a track has distinct cameras)
      for (int o = S->lm_seg[i]; o < S->lm_seg[i + 1]; ++o) fresh += stamp[S->cam_of[o]] != tile_id;
      const bool new_prob = i > 0 && S->lm_prob[i] != S->lm_prob[i - 1];
      // a piece of a long track has a tile of its own
      const bool piece = S->lm_long[i] >= 0 || (i > 0 && S->lm_long[i - 1] >= 0);
      if (tile_lms > 0 && (new_prob || piece || tile_obs + k > kTileObs ||
                           tile_lms + 1 > kTileLms || tile_cams + fresh > kTileSlots)) {
        S->tile_lm0.push_back(i);
        tile_obs = 0;
        tile_lms = 0;
        tile_cams = 0;
        ++tile_id;
        fresh = k;
      }
      for (int o = S->lm_seg[i]; o < S->lm_seg[i + 1]; ++o) stamp[S->cam_of[o]] = tile_id;
      tile_obs += k;
      tile_lms += 1;
      tile_cams += fresh;
    }
    S->tile_lm0.push_back(n_int);
  }
  S->n_tiles = (int)S->tile_lm0.size() - 1;
  S->long_tile0.assign(S->n_long, 0);
  for (int t = 0; t < S->n_tiles; ++t) {
    const int j = S->lm_long[S->tile_lm0[t]];
    if (j >= 0 && S->tile_lm0[t] == S->long_first[j]) S->long_tile0[j] = t;
  }
  S->tile_off.assign(n_probs + 1, 0);
  for (int t = 0; t < S->n_tiles; ++t) S->tile_off[S->lm_prob[S->tile_lm0[t]] + 1]++;
  for (int p = 0; p < n_probs; ++p) S->tile_off[p + 1] += S->tile_off[p];

  // Slots: distinct cameras per tile, ascending; per observation its slot and its position in
  // the tile's camera-sorted order (stable in landmark order).
  S->obs_meta.assign(n_obs, 0);
  S->tile_slot0.assign(S->n_tiles + 1, 0);
  S->slot_cam.clear();
  S->slot_beg.clear();
  S->max_slots_per_tile = 0;
  std::vector<int32_t> local;  // observation offsets within the tile
  for (int t = 0; t < S->n_tiles; ++t) {
    int o0 = S->lm_seg[S->tile_lm0[t]], o1 = S->lm_seg[S->tile_lm0[t + 1]];
    int n = o1 - o0;
    local.resize(n);
    std::iota(local.begin(), local.end(), 0);
    std::stable_sort(local.begin(), local.end(),
                     [&](int32_t a, int32_t b) { return S->cam_of[o0 + a] < S->cam_of[o0 + b]; });
    int slot = -1, prev_cam = -1;
    for (int p = 0; p < n; ++p) {
      int o = o0 + local[p];
      int c = S->cam_of[o];
      if (c != prev_cam) {
        ++slot;
        prev_cam = c;
        S->slot_cam.push_back(c);
        S->slot_beg.push_back((uint16_t)p);
      }
      S->obs_meta[o] = (uint16_t)(p | (slot << 8));
    }
    int ns = slot + 1;
    S->max_slots_per_tile = std::max(S->max_slots_per_tile, ns);
    S->tile_slot0[t + 1] = S->tile_slot0[t] + ns;
  }
  S->n_slots = S->tile_slot0[S->n_tiles];
  S->tile_desc.assign((size_t)S->n_tiles * 8, 0);
  size_t rec_bytes = 0;
  for (int t = 0; t < S->n_tiles; ++t) {
    int32_t* d = &S->tile_desc[(size_t)t * 8];
    d[0] = S->tile_lm0[t];
    d[1] = S->tile_lm0[t + 1] - S->tile_lm0[t];
    d[2] = S->lm_seg[S->tile_lm0[t]];
    d[3] = S->lm_seg[S->tile_lm0[t + 1]] - d[2];
    d[4] = S->tile_slot0[t];
    d[5] = S->tile_slot0[t + 1] - S->tile_slot0[t];
    d[6] = (int32_t)(rec_bytes / 16);
    d[7] = S->lm_prob[S->tile_lm0[t]];
    rec_bytes += (size_t)tile_rec_layout(d[3], d[5], d[1]).bytes;
  }
  if (rec_bytes / 16 > (size_t)INT32_MAX) return "too many tiles for the tile records";

  // Camera -> slots (CSR), slots in tile order.
  S->cam_slot_ptr.assign(n_cams + 1, 0);
  for (int s = 0; s < S->n_slots; ++s) S->cam_slot_ptr[S->slot_cam[s] + 1]++;
  for (int c = 0; c < n_cams; ++c) S->cam_slot_ptr[c + 1] += S->cam_slot_ptr[c];
  S->cam_slot_list.assign(S->n_slots, 0);
  std::vector<int32_t> fill(S->cam_slot_ptr.begin(), S->cam_slot_ptr.end() - 1);
  for (int s = 0; s < S->n_slots; ++s) S->cam_slot_list[fill[S->slot_cam[s]]++] = s;
  S->slot_row.assign(S->n_slots, 0);
  for (int r = 0; r < S->n_slots; ++r) S->slot_row[S->cam_slot_list[r]] = r;

  // Per-tile records (copies of the index data above, grouped per tile).
  S->tile_rec.assign(rec_bytes, 0);
  for (int t = 0; t < S->n_tiles; ++t) {
    const int32_t* d = &S->tile_desc[(size_t)t * 8];
    const int L0 = d[0], nl = d[1], o0 = d[2], n = d[3], S0 = d[4], ns = d[5];
    const TileRecLayout g = tile_rec_layout(n, ns, nl);
    uint8_t* base = &S->tile_rec[(size_t)d[6] * 16];
    uint16_t* meta = reinterpret_cast<uint16_t*>(base + g.meta);
    uint8_t* olm = base + g.olm;
    uint16_t* sbeg = reinterpret_cast<uint16_t*>(base + g.sbeg);
    uint16_t* sseg = reinterpret_cast<uint16_t*>(base + g.sseg);
    int32_t* srow = reinterpret_cast<int32_t*>(base + g.srow);
    int32_t* scam = reinterpret_cast<int32_t*>(base + g.scam);
    for (int i = 0; i < n; ++i) meta[i] = S->obs_meta[o0 + i];
    for (int l = 0; l < nl; ++l)
      for (int o = S->lm_seg[L0 + l]; o < S->lm_seg[L0 + l + 1]; ++o) olm[o - o0] = (uint8_t)l;
    for (int s = 0; s < ns; ++s) {
      sbeg[s] = S->slot_beg[S0 + s];
      srow[s] = S->slot_row[S0 + s];
      scam[s] = S->slot_cam[S0 + s];
    }
    for (int l = 0; l <= nl; ++l) sseg[l] = (uint16_t)(S->lm_seg[L0 + l] - o0);
  }
  return "";
}

std::string build_series_schedule(const Schedule& S, int target, int tail, SerSchedule* Q,
                                  int slot_cap) {
  if (target < 1) return "the group size must be >= 1";
  if (slot_cap < 1 || slot_cap > kGroupSlots) return "the group slot cap must be in [1, 256]";
  if (tail < 0 || tail > 64) return "the tail split must be in [0, 64]";
  Q->target = target;
  Q->tail = tail;
  std::vector<int32_t> gnat;   // groups in landmark order: [8] each (see SerSchedule::group)
  std::vector<int32_t> gcams;  // the groups' distinct cameras, ascending, concatenated
  Q->chunk.clear();
  Q->rec.clear();
  std::vector<int32_t> stamp(S.n_cams, -1);  // range that last counted the camera
  std::vector<int32_t> gslot_of(S.n_cams, -1);
  std::vector<int32_t> local;
  struct Range {
    int l, le;
    bool long_track;  // the pieces of one long track (a long group)
  };
  std::vector<Range> ranges;  // one problem's groups as landmark ranges
  // a landmark seen by more than slot_cap cameras (possible when slot_cap < kChunkObs) cannot
  // share a group's slots: like a long track's pieces it becomes a group of its own, whose chunk
  // keeps slots of its own (the long-group body), so that every other group stays within the cap
  std::vector<char> wide(S.n_lms_int, 0);
  for (int l = 0; l < S.n_lms_int; ++l) {
    if (S.lm_long[l] >= 0 || S.lm_seg[l + 1] - S.lm_seg[l] <= slot_cap) continue;
    int ncam = 0;
    for (int o = S.lm_seg[l]; o < S.lm_seg[l + 1]; ++o)
      if (stamp[S.cam_of[o]] != l) {
        stamp[S.cam_of[o]] = l;
        ++ncam;
      }
    wide[l] = ncam > slot_cap;
  }
  std::fill(stamp.begin(), stamp.end(), -1);
  int n_groups = 0, rid = 0, n_long_groups = 0;
  int next_tag = -2;  // marks of gslot_of while a slot set is collected (slots are >= 0)
  for (int p = 0; p < S.n_probs; ++p) {
    // the problem's observed landmarks (unobserved ones sort last within their problem)
    const int l0 = S.lm_off_int[p];
    int l1 = S.lm_off_int[p + 1];
    while (l1 > l0 && S.lm_seg[l1] == S.lm_seg[l1 - 1]) --l1;
    const int64_t o_beg = S.lm_seg[l0], n_p = (int64_t)S.lm_seg[l1] - o_beg;
    if (n_p == 0) continue;
    const int64_t ng = (n_p + target - 1) / target;
    int64_t k_next = 1;  // index of the next balanced boundary
    ranges.clear();
    for (int l = l0; l < l1;) {
      if (S.lm_long[l] >= 0 || wide[l]) {
        // a long track: its pieces form one group of their own (a wide landmark: one piece)
        const int le = S.lm_long[l] >= 0 ? l + S.long_np[S.lm_long[l]] : l + 1;
        ranges.push_back({l, le, true});
        const int64_t done = (int64_t)S.lm_seg[le] - o_beg;
        while (k_next < ng && done * ng >= k_next * n_p) ++k_next;
        l = le;
        continue;
      }
      // one range: landmarks [l, le), ending at the balanced boundary k_next * n_p / ng
      // (observations from the problem's start), before a long track, or before its cameras
      // would exceed slot_cap
      const int r = rid++;
      int le = l, ncam = 0;
      while (le < l1) {
        if (S.lm_long[le] >= 0 || wide[le]) break;
        const int a = S.lm_seg[le], b = S.lm_seg[le + 1];
        int fresh = 0;
        for (int o = a; o < b; ++o) fresh += stamp[S.cam_of[o]] != r;
        if (le > l && ncam + fresh > slot_cap) break;
        for (int o = a; o < b; ++o) {
          if (stamp[S.cam_of[o]] != r) {
            stamp[S.cam_of[o]] = r;
            ++ncam;
          }
        }
        ++le;
        const int64_t done = (int64_t)S.lm_seg[le] - o_beg;
        if (done * ng >= k_next * n_p) {
          while (k_next < ng && done * ng >= k_next * n_p) ++k_next;
          break;
        }
      }
      // tail split: the range's last eighth of observations becomes `tail` small ranges
      const int64_t n_r = (int64_t)S.lm_seg[le] - S.lm_seg[l];
      if (tail > 0 && n_r >= 2 * kChunkObs) {
        const int64_t head_end = S.lm_seg[l] + n_r - n_r / 8;
        int lh = l + 1;
        while (lh < le && S.lm_seg[lh] < head_end) ++lh;
        ranges.push_back({l, lh, false});
        const int64_t t0 = S.lm_seg[lh], n_t = (int64_t)S.lm_seg[le] - t0;
        int lt = lh;
        for (int k = 1; k <= tail && lt < le; ++k) {
          int lte = lt + 1;
          while (lte < le && ((int64_t)S.lm_seg[lte] - t0) * tail < k * n_t) ++lte;
          if (k == tail) lte = le;
          ranges.push_back({lt, lte, false});
          lt = lte;
        }
      } else {
        ranges.push_back({l, le, false});
      }
      l = le;
    }
    for (const auto& rg : ranges) {
      const int l = rg.l, le = rg.le;
      const int g = n_groups++;
      const int gs0 = (int)gcams.size();
      // The group's distinct cameras, ascending, are its slots.  A long group's chunks (one
      // piece each) have slots of their own instead: each chunk's distinct cameras, ascending,
      // from slot base d[7] on (code and clist hold chunk-relative slots).
      auto add_slots = [&](int oa, int ob, int tag) {
        const int s0 = (int)gcams.size();
        for (int o = oa; o < ob; ++o) {
          const int c = S.cam_of[o];
          if (gslot_of[c] != tag) {
            gslot_of[c] = tag;
            gcams.push_back(c);
          }
        }
        std::sort(gcams.begin() + s0, gcams.end());
        for (int s = s0; s < (int)gcams.size(); ++s) gslot_of[gcams[s]] = s - s0;
        return s0 - gs0;
      };
      if (!rg.long_track) add_slots(S.lm_seg[l], S.lm_seg[le], next_tag--);
      // chunks: whole landmarks, at most kChunkObs observations (a long group: one piece each)
      const int c0 = (int)(Q->chunk.size() / 8);
      int lc = l;
      while (lc < le) {
        int lce = lc;
        if (rg.long_track)
          lce = lc + 1;
        else
          while (lce < le && S.lm_seg[lce + 1] - S.lm_seg[lc] <= kChunkObs) ++lce;
        if (lce == lc) return "a landmark has more observations than a chunk holds";
        const int o0 = S.lm_seg[lc], n = S.lm_seg[lce] - o0, nl = lce - lc;
        const int sbase = rg.long_track
                              ? add_slots(o0, o0 + n, next_tag--)
                              : 0;
        local.resize(n);
        for (int i = 0; i < n; ++i) local[i] = i;
        std::stable_sort(local.begin(), local.end(), [&](int32_t x, int32_t y) {
          return S.cam_of[o0 + x] < S.cam_of[o0 + y];
        });
        std::vector<uint32_t> code(n), clist;
        int prev = -1;
        for (int q = 0; q < n; ++q) {
          const int i = local[q], cam = S.cam_of[o0 + i];
          if (cam != prev) {
            clist.push_back((uint32_t)gslot_of[cam] | ((uint32_t)q << 8));
            prev = cam;
          }
          clist.back() += 1u << 16;  // one more row
          code[i] = (uint32_t)q | ((uint32_t)gslot_of[cam] << 8) |
                    ((uint32_t)(S.lm_of[o0 + i] - lc) << 16);
        }
        std::stable_sort(clist.begin(), clist.end(),
                         [](uint32_t x, uint32_t y) { return (x >> 16) > (y >> 16); });
        const int ns = (int)clist.size();
        const ChunkRecLayout L = chunk_rec_layout(n, nl, ns);
        const size_t off = Q->rec.size();
        if (off / 16 > (size_t)INT32_MAX) return "too many chunks for the chunk records";
        Q->rec.resize(off + L.bytes, 0);
        uint8_t* base = Q->rec.data() + off;
        std::memcpy(base + L.code, code.data(), 4 * (size_t)n);
        uint16_t* sseg = reinterpret_cast<uint16_t*>(base + L.sseg);
        for (int j = 0; j <= nl; ++j) sseg[j] = (uint16_t)(S.lm_seg[lc + j] - o0);
        std::memcpy(base + L.clist, clist.data(), 4 * (size_t)ns);
        const int32_t d[8] = {o0, n, lc, nl, ns, (int32_t)(off / 16), g, sbase};
        Q->chunk.insert(Q->chunk.end(), d, d + 8);
        lc = lce;
      }
      const int nc = (int)(Q->chunk.size() / 8) - c0;
      const int ns_g = (int)gcams.size() - gs0;
      const int32_t gd[8] = {c0, nc, gs0, ns_g, S.lm_seg[le] - S.lm_seg[l], p,
                             rg.long_track ? 1 : 0, 0};
      n_long_groups += rg.long_track ? 1 : 0;
      gnat.insert(gnat.end(), gd, gd + 8);
    }
  }
  Q->n_groups = n_groups;
  Q->n_long_groups = n_long_groups;
  Q->n_chunks = (int)(Q->chunk.size() / 8);
  Q->n_gslots = (int)gcams.size();
  Q->gslot_cam = gcams;
  Q->max_group_slots = 0;
  for (int g = 0; g < n_groups; ++g) Q->max_group_slots = std::max(Q->max_group_slots, gnat[8 * g + 3]);
  // camera-major rows: camera c's rows are its group slots in landmark (group) order
  Q->cam_ptr.assign(S.n_cams + 1, 0);
  for (int c : gcams) Q->cam_ptr[c + 1]++;
  for (int c = 0; c < S.n_cams; ++c) Q->cam_ptr[c + 1] += Q->cam_ptr[c];
  Q->prob_ncam.assign(S.n_probs, 0);
  for (int p = 0; p < S.n_probs; ++p)
    for (int c = S.cam_off[p]; c < S.cam_off[p + 1]; ++c)
      Q->prob_ncam[p] += Q->cam_ptr[c + 1] > Q->cam_ptr[c] ? 1 : 0;
  std::vector<int32_t> fill(Q->cam_ptr.begin(), Q->cam_ptr.end() - 1);
  Q->gslot_row.assign(Q->n_gslots, 0);
  for (int s = 0; s < Q->n_gslots; ++s) Q->gslot_row[s] = fill[gcams[s]]++;
  // ticket order: decreasing observation count (longest first), ties in landmark order
  std::vector<int32_t> ord(n_groups);
  for (int g = 0; g < n_groups; ++g) ord[g] = g;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int32_t x, int32_t y) { return gnat[8 * x + 4] > gnat[8 * y + 4]; });
  Q->group.assign((size_t)n_groups * 8, 0);
  std::vector<int32_t> ticket(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    std::memcpy(&Q->group[(size_t)i * 8], &gnat[(size_t)ord[i] * 8], 8 * sizeof(int32_t));
    ticket[ord[i]] = i;
  }
  // each chunk names its group by ticket
  for (int c = 0; c < Q->n_chunks; ++c) Q->chunk[(size_t)c * 8 + 6] = ticket[Q->chunk[(size_t)c * 8 + 6]];
  return "";
}

int series_auto_target(int64_t n_obs, int G) {
  const int64_t t = G > 0 ? (n_obs + G - 1) / G : n_obs;
  return (int)std::min<int64_t>(std::max<int64_t>(t, kChunkObs), INT32_MAX);
}

void build_cam_schedule(const std::vector<int32_t>& cam_ptr, int n_cams, CamSchedule* cs) {
  cs->cam_item.assign(n_cams + 1, 0);
  cs->item_q.clear();
  for (int c = 0; c < n_cams; ++c) {
    const int r0 = cam_ptr[c], r1 = cam_ptr[c + 1];
    const int k = cam_chunks(r1 - r0), C = cam_chunk_rows(r1 - r0);
    for (int j = 0; j < k; ++j) {
      cs->item_q.push_back(std::min(r0 + j * C, r1));
      cs->item_q.push_back(std::min(r0 + (j + 1) * C, r1));
    }
    cs->cam_item[c + 1] = cs->cam_item[c] + k;
  }
}

void build_cam_rounds(const CamSchedule& cs, int n_cams, int G, CamRoundList* out) {
  const int total = cs.cam_item[n_cams];
  int biggest = 1;
  for (int c = 0; c < n_cams; ++c) biggest = std::max(biggest, cs.cam_item[c + 1] - cs.cam_item[c]);
  int max_items = (total + G - 1) / G;
  max_items = std::min(kRoundItems, std::max(max_items, biggest));
  out->round_cam.assign(1, 0);
  out->round_item.assign(1, 0);
  int in_round = 0;
  for (int c = 0; c < n_cams; ++c) {
    const int k = cs.cam_item[c + 1] - cs.cam_item[c];
    if (c > out->round_cam.back() && in_round + k > max_items) {
      out->round_cam.push_back(c);
      out->round_item.push_back(cs.cam_item[c]);
      in_round = 0;
    }
    in_round += k;
  }
  out->round_cam.push_back(n_cams);
  out->round_item.push_back(total);
  const int R = (int)out->round_cam.size() - 1;
  out->block_round.assign(G + 1, 0);
  for (int b = 0; b <= G; ++b) out->block_round[b] = (int)(((int64_t)b * R) / G);
}

}  // namespace poba
