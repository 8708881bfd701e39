// Host check of the library's tile schedule (no GPU; test infrastructure for
// tests/test_schedule_cpu.py).  Reads one problem's (or one batch's) observation indices from a
// file, builds the schedule and the camera rounds for a grid of G blocks, and verifies the
// properties the kernels rely on.  Prints "ok ..." or the first violated property.
//
// Input (little-endian int32): P, n_cams, n_lms, n_obs, G, cam_off[P + 1], lm_off[P + 1],
// cam_idx[n_obs], lm_idx[n_obs].
#include <cstdio>
#include <algorithm>
#include <set>
#include <string>
#include <vector>

#include "poba_internal.cuh"

using namespace poba;

#define CHECK(cond, ...)                 \
  do {                                   \
    if (!(cond)) {                       \
      std::printf("FAIL: " __VA_ARGS__); \
      std::printf("\n");                 \
      return 1;                          \
    }                                    \
  } while (0)

static bool read_ints(FILE* f, int32_t* p, size_t n) { return std::fread(p, 4, n, f) == n; }

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[5];
  if (!read_ints(f, hdr, 5)) return 2;
  const int P = hdr[0], nc = hdr[1], nl = hdr[2], no = hdr[3], G = hdr[4];
  std::vector<int32_t> cam_off(P + 1), lm_off(P + 1), cam(no), lm(no);
  if (!read_ints(f, cam_off.data(), P + 1) || !read_ints(f, lm_off.data(), P + 1) ||
      !read_ints(f, cam.data(), no) || !read_ints(f, lm.data(), no))
    return 2;
  std::fclose(f);

  Schedule S;
  const std::string why = build_schedule(nc, nl, no, cam.data(), lm.data(), P,
                                         P > 1 ? cam_off.data() : nullptr,
                                         P > 1 ? lm_off.data() : nullptr, &S);
  CHECK(why.empty(), "build_schedule rejected the input: %s", why.c_str());

  const int nli = S.n_lms_int;  // internal landmarks: long tracks count once per piece
  // observations: a permutation of the caller's, sorted by (internal landmark, camera)
  std::vector<char> seen(no, 0);
  for (int o = 0; o < no; ++o) {
    const int64_t q = S.obs_order[o];
    CHECK(q >= 0 && q < no && !seen[q], "obs_order is not a permutation at %d", o);
    seen[q] = 1;
    CHECK(S.cam_of[o] == cam[q], "cam_of[%d] is not the caller's camera", o);
    CHECK(S.lm_of[o] >= 0 && S.lm_of[o] < nli && S.lm_order[S.lm_of[o]] == lm[q] &&
              S.lm_of[o] >= S.lm_rank[lm[q]],
          "lm_of[%d] is not (a piece of) the internal landmark", o);
    if (o > 0) {
      CHECK(S.lm_of[o] > S.lm_of[o - 1] ||
                (S.lm_of[o] == S.lm_of[o - 1] && S.cam_of[o] >= S.cam_of[o - 1]),
            "observations %d, %d out of (landmark, camera) order", o - 1, o);
    }
  }
  for (int l = 0; l < nli; ++l)
    for (int o = S.lm_seg[l]; o < S.lm_seg[l + 1]; ++o)
      CHECK(S.lm_of[o] == l, "lm_seg of landmark %d holds observation %d of another", l, o);
  CHECK(S.lm_seg[0] == 0 && S.lm_seg[nli] == no, "lm_seg does not cover the observations");

  // long tracks: a landmark of more than kTileObs observations is split into consecutive pieces
  // of near-equal size (at most kTileObs), in camera order, each alone in its tile
  {
    std::vector<int> cnt(nl, 0);
    for (int o = 0; o < no; ++o) cnt[lm[o]]++;
    int n_long = 0, extra = 0;
    for (int l = 0; l < nl; ++l)
      if (cnt[l] > kTileObs) {
        ++n_long;
        extra += (cnt[l] + kTileObs - 1) / kTileObs - 1;
      }
    CHECK(S.n_long == n_long && nli == nl + extra, "%d long tracks, %d internal landmarks", S.n_long,
          nli);
    std::vector<int> long_of(nli, -1);
    for (int j = 0; j < S.n_long; ++j) {
      const int e0 = S.long_first[j], np = S.long_np[j], l = S.lm_order[e0];
      CHECK(np >= 2 && np == (cnt[l] + kTileObs - 1) / kTileObs, "long track %d has %d pieces", j, np);
      CHECK(S.lm_rank[l] == e0, "long track %d: the caller's landmark maps to its first piece", j);
      CHECK(S.lm_seg[e0 + np] - S.lm_seg[e0] == cnt[l], "long track %d observation count", j);
      int lo = 1 << 30, hi = 0;
      for (int q = 0; q < np; ++q) {
        const int e = e0 + q, k = S.lm_seg[e + 1] - S.lm_seg[e], t = S.long_tile0[j] + q;
        CHECK(S.lm_order[e] == l && S.lm_long[e] == j, "long track %d piece %d", j, q);
        CHECK(t < S.n_tiles && S.tile_lm0[t] == e && S.tile_lm0[t + 1] == e + 1,
              "long track %d piece %d is not alone in tile %d", j, q, t);
        long_of[e] = j;
        lo = std::min(lo, k);
        hi = std::max(hi, k);
      }
      CHECK(hi <= kTileObs && hi - lo <= 1, "long track %d pieces of %d .. %d observations", j, lo, hi);
    }
    for (int e = 0; e < nli; ++e) {
      CHECK(S.lm_long[e] == long_of[e], "lm_long[%d]", e);
      CHECK(S.lm_seg[e + 1] - S.lm_seg[e] <= kTileObs, "landmark %d exceeds a tile", e);
    }
  }

  // tiles: whole landmarks of one problem within the caps; slots = the tile's cameras ascending
  CHECK(S.tile_lm0.front() == 0 && S.tile_lm0.back() == nli, "tiles do not cover the landmarks");
  std::vector<int> slot_count_of_cam(nc, 0);
  for (int t = 0; t < S.n_tiles; ++t) {
    const int L0 = S.tile_lm0[t], L1 = S.tile_lm0[t + 1];
    CHECK(L1 > L0, "tile %d is empty", t);
    const int o0 = S.lm_seg[L0], n = S.lm_seg[L1] - o0;
    const int nlt = L1 - L0;
    std::set<int> cams;
    for (int o = o0; o < o0 + n; ++o) cams.insert(S.cam_of[o]);
    CHECK(nlt <= kTileLms, "tile %d holds %d landmarks", t, nlt);
    CHECK(n <= kTileObs, "tile %d holds %d observations", t, n);
    CHECK((int)cams.size() <= kTileSlots || nlt == 1, "tile %d holds %d cameras", t,
          (int)cams.size());
    for (int l = L0 + 1; l < L1; ++l)
      CHECK(S.lm_prob[l] == S.lm_prob[L0], "tile %d holds two problems", t);
    const int s0 = S.tile_slot0[t], ns = S.tile_slot0[t + 1] - s0;
    CHECK(ns == (int)cams.size(), "tile %d has %d slots for %d cameras", t, ns, (int)cams.size());
    int s = 0;
    for (int c : cams) {
      CHECK(S.slot_cam[s0 + s] == c, "tile %d slot %d is not its %d-th camera", t, s, s);
      ++slot_count_of_cam[c];
      ++s;
    }
    // observation codes: the slot of its camera, and positions that sort the tile by
    // (camera, landmark order)
    std::vector<int> at(n, -1);
    for (int o = o0; o < o0 + n; ++o) {
      const int pos = S.obs_meta[o] & 0xff, sl = S.obs_meta[o] >> 8;
      CHECK(sl < ns && S.slot_cam[s0 + sl] == S.cam_of[o], "observation %d has a wrong slot", o);
      CHECK(pos < n && at[pos] < 0, "observation %d has a repeated position", o);
      at[pos] = o;
    }
    for (int p = 1; p < n; ++p) {
      const int a = at[p - 1], b = at[p];
      CHECK(S.cam_of[a] < S.cam_of[b] || (S.cam_of[a] == S.cam_of[b] && a < b),
            "tile %d positions %d, %d are not in (camera, landmark) order", t, p - 1, p);
    }
    for (int sl = 0; sl < ns; ++sl) {
      const int p = S.slot_beg[s0 + sl];
      CHECK(p < n && S.cam_of[at[p]] == S.slot_cam[s0 + sl] &&
                (p == 0 || S.cam_of[at[p - 1]] != S.slot_cam[s0 + sl]),
            "tile %d slot %d does not start at its camera's first position", t, sl);
    }
  }

  // camera-major rows: each camera's slots are contiguous rows, in tile order
  CHECK(S.cam_slot_ptr[0] == 0 && S.cam_slot_ptr[nc] == S.n_slots, "camera rows do not cover slots");
  std::vector<char> row_seen(S.n_slots, 0);
  for (int s = 0; s < S.n_slots; ++s) {
    const int r = S.slot_row[s];
    CHECK(r >= 0 && r < S.n_slots && !row_seen[r], "slot_row is not a permutation at %d", s);
    row_seen[r] = 1;
    CHECK(S.cam_slot_list[r] == s, "cam_slot_list is not the inverse of slot_row at %d", r);
    const int c = S.slot_cam[s];
    CHECK(r >= S.cam_slot_ptr[c] && r < S.cam_slot_ptr[c + 1], "slot %d's row is not its camera's", s);
  }
  for (int c = 0; c < nc; ++c) {
    CHECK(S.cam_slot_ptr[c + 1] - S.cam_slot_ptr[c] == slot_count_of_cam[c],
          "camera %d has a wrong row count", c);
    for (int r = S.cam_slot_ptr[c] + 1; r < S.cam_slot_ptr[c + 1]; ++r)
      CHECK(S.cam_slot_list[r] > S.cam_slot_list[r - 1], "camera %d's rows are not in tile order", c);
  }

  // series schedule for a grid of G blocks: groups of whole landmarks of one problem, balanced
  // by observation count, at most `cap` cameras; chunks of whole landmarks; records
  SerSchedule Q;
  const int target = series_auto_target(no, G);
  const int tail = G % 3;  // exercise the tail split on some grids
  const int cap = G % 2 ? kGroupSlotsF64 : kGroupSlots;  // both precisions' slot caps
  const std::string qwhy = build_series_schedule(S, target, tail, &Q, cap);
  CHECK(qwhy.empty(), "build_series_schedule failed: %s", qwhy.c_str());
  CHECK((int)Q.group.size() == 8 * Q.n_groups && (int)Q.chunk.size() == 8 * Q.n_chunks,
        "series descriptor sizes");
  std::vector<int> chunk_group(Q.n_chunks, -1);
  int n_lg = 0, n_wide = 0;
  std::vector<int> group_of_slot(Q.n_gslots, -1);
  std::vector<int> slot_key(Q.n_gslots, -1);  // landmark order: the chunk its rows start in
  for (int i = 0; i < Q.n_groups; ++i) {
    const int32_t* g = &Q.group[8 * (size_t)i];
    if (i > 0) CHECK(g[4] <= Q.group[8 * (size_t)(i - 1) + 4], "groups not in decreasing size order at %d", i);
    CHECK(g[1] >= 1 && g[0] >= 0 && g[0] + g[1] <= Q.n_chunks, "group %d chunk range", i);
    const bool lg = g[6] != 0;  // a long group: a long track's pieces or one wide landmark
    n_lg += lg ? 1 : 0;
    CHECK(g[3] >= 1 && (lg || g[3] <= cap) && g[2] >= 0 && g[2] + g[3] <= Q.n_gslots,
          "group %d slot range (%d slots)", i, g[3]);
    int obs = 0;
    std::set<int> cams;
    int s = g[2];
    for (int c = g[0]; c < g[0] + g[1]; ++c) {
      CHECK(chunk_group[c] < 0, "chunk %d in two groups", c);
      chunk_group[c] = i;
      const int32_t* d = &Q.chunk[8 * (size_t)c];
      CHECK(d[6] == i, "chunk %d names group %d, not %d", c, d[6], i);
      obs += d[1];
      if (c > g[0]) CHECK(d[2] == Q.chunk[8 * (size_t)(c - 1) + 2] + Q.chunk[8 * (size_t)(c - 1) + 3],
                          "group %d chunks are not consecutive landmarks", i);
      for (int o = d[0]; o < d[0] + d[1]; ++o) {
        cams.insert(S.cam_of[o]);
        CHECK(S.lm_prob[S.lm_of[o]] == g[5], "group %d holds another problem's observation", i);
      }
      for (int l = d[2]; l < d[2] + d[3]; ++l) {
        const int j = S.lm_long[l];
        CHECK(lg || j < 0, "group %d: a piece of a long track in a plain group", i);
        if (lg && j >= 0) {
          CHECK(d[3] == 1 && l == S.long_first[j] + (c - g[0]) && g[1] == S.long_np[j],
                "long group %d chunk %d is not piece %d of its track", i, c, c - g[0]);
        } else if (lg) {
          // a landmark seen by more cameras than the slot cap: a group of one piece
          std::set<int> lc;
          for (int o = S.lm_seg[l]; o < S.lm_seg[l + 1]; ++o) lc.insert(S.cam_of[o]);
          CHECK(d[3] == 1 && g[1] == 1 && (int)lc.size() > cap,
                "long group %d is neither a long track nor one landmark wider than the cap", i);
          ++n_wide;
        }
      }
      if (lg) {
        // the chunk's slots: its cameras, ascending, from slot base d[7]
        std::set<int> cc;
        for (int o = d[0]; o < d[0] + d[1]; ++o) cc.insert(S.cam_of[o]);
        CHECK(g[2] + d[7] == s, "long group %d chunk %d slot base", i, c);
        for (int cam : cc) {
          CHECK(Q.gslot_cam[s] == cam, "long group %d chunk %d slot is not its camera", i, c);
          CHECK(group_of_slot[s] < 0, "group slot %d shared", s);
          group_of_slot[s] = i;
          slot_key[s] = c;
          ++s;
        }
      } else {
        CHECK(d[7] == 0, "chunk %d of plain group %d has a slot base", c, i);
      }
    }
    CHECK(obs == g[4], "group %d observation count", i);
    if (!lg) {
      CHECK((int)cams.size() == g[3], "group %d has %d cameras but %d slots", i, (int)cams.size(), g[3]);
      for (int cam : cams) {  // ascending
        CHECK(Q.gslot_cam[s] == cam, "group %d slot %d is not its %d-th camera", i, s - g[2], s - g[2]);
        CHECK(group_of_slot[s] < 0, "group slot %d shared", s);
        group_of_slot[s] = i;
        slot_key[s] = g[0];
        ++s;
      }
    }
    CHECK(s == g[2] + g[3], "group %d slot count", i);
  }
  CHECK(n_lg == Q.n_long_groups, "long group count %d, schedule says %d", n_lg, Q.n_long_groups);
  {
    // every landmark wider than the cap (and not a long track) has a group of its own
    int wide = 0;
    for (int l = 0; l < S.n_lms_int; ++l) {
      if (S.lm_long[l] >= 0) continue;
      std::set<int> lc;
      for (int o = S.lm_seg[l]; o < S.lm_seg[l + 1]; ++o) lc.insert(S.cam_of[o]);
      wide += (int)lc.size() > cap ? 1 : 0;
    }
    CHECK(wide == n_wide, "%d landmarks wider than the cap, %d wide groups", wide, n_wide);
  }
  // chunks in landmark order cover every observation once
  {
    int next_o = 0;
    for (int c = 0; c < Q.n_chunks; ++c) {
      const int32_t* d = &Q.chunk[8 * (size_t)c];
      const int o0 = d[0], n = d[1], L0 = d[2], nl = d[3], ns = d[4];
      CHECK(chunk_group[c] >= 0, "chunk %d in no group", c);
      CHECK(n >= 1 && n <= kChunkObs && nl >= 1, "chunk %d size (%d obs, %d landmarks)", c, n, nl);
      CHECK(o0 == S.lm_seg[L0] && o0 + n == S.lm_seg[L0 + nl], "chunk %d is not whole landmarks", c);
      CHECK(o0 >= next_o, "chunks overlap at %d", c);
      for (int o = next_o; o < o0; ++o) CHECK(false, "observation %d is in no chunk", o);
      next_o = o0 + n;
      const int32_t* g = nullptr;
      for (int i = 0; i < Q.n_groups; ++i)
        if (Q.group[8 * (size_t)i] <= c && c < Q.group[8 * (size_t)i] + Q.group[8 * (size_t)i + 1])
          g = &Q.group[8 * (size_t)i];
      const ChunkRecLayout L = chunk_rec_layout(n, nl, ns);
      CHECK((size_t)d[5] * 16 + L.bytes <= Q.rec.size(), "chunk %d record out of range", c);
      const uint8_t* base = Q.rec.data() + (size_t)d[5] * 16;
      const uint32_t* code = reinterpret_cast<const uint32_t*>(base + L.code);
      const uint16_t* sseg = reinterpret_cast<const uint16_t*>(base + L.sseg);
      const uint32_t* clist = reinterpret_cast<const uint32_t*>(base + L.clist);
      for (int j = 0; j <= nl; ++j)
        CHECK(sseg[j] == S.lm_seg[L0 + j] - o0, "chunk %d segment %d", c, j);
      std::vector<int> at(n, -1);
      for (int i = 0; i < n; ++i) {
        const int pos = code[i] & 0xff, gs = (code[i] >> 8) & 0xff, lm = (code[i] >> 16) & 0xff;
        CHECK((code[i] >> 24) == 0, "chunk %d code high bits", c);
        CHECK(pos < n && at[pos] < 0, "chunk %d positions are not a permutation", c);
        at[pos] = i;
        CHECK(d[7] + gs < g[3] && Q.gslot_cam[g[2] + d[7] + gs] == S.cam_of[o0 + i],
              "chunk %d obs %d group slot", c, i);
        CHECK(L0 + lm == S.lm_of[o0 + i], "chunk %d obs %d landmark", c, i);
      }
      for (int q = 1; q < n; ++q) {
        const int a = at[q - 1], b = at[q];
        CHECK(S.cam_of[o0 + a] < S.cam_of[o0 + b] || (S.cam_of[o0 + a] == S.cam_of[o0 + b] && a < b),
              "chunk %d positions are not in (camera, landmark) order", c);
      }
      // chunk slots: each camera's run of positions once, longest first (ties by position)
      std::vector<int> run_beg, run_len, run_cam;
      for (int q = 0; q < n; ++q) {
        const int cam = S.cam_of[o0 + at[q]];
        if (q == 0 || cam != S.cam_of[o0 + at[q - 1]]) {
          run_beg.push_back(q);
          run_len.push_back(0);
          run_cam.push_back(cam);
        }
        run_len.back()++;
      }
      CHECK((int)run_beg.size() == ns, "chunk %d slot count", c);
      std::vector<char> used(ns, 0);
      for (int j = 0; j < ns; ++j) {
        const int gs = clist[j] & 0xff, beg = (clist[j] >> 8) & 0xff, len = (int)(clist[j] >> 16);
        if (j > 0) {
          const int lp = (int)(clist[j - 1] >> 16), bp = (clist[j - 1] >> 8) & 0xff;
          CHECK(len < lp || (len == lp && beg > bp), "chunk %d slots not longest first", c);
        }
        int r = -1;
        for (int k = 0; k < ns; ++k)
          if (run_beg[k] == beg) r = k;
        CHECK(r >= 0 && !used[r] && run_len[r] == len && Q.gslot_cam[g[2] + d[7] + gs] == run_cam[r],
              "chunk %d slot %d", c, j);
        used[r] = 1;
      }
    }
    for (int o = next_o; o < no; ++o) CHECK(false, "observation %d is in no chunk", o);
  }
  // balance: groups of a single problem differ by at most one track plus the size split
  if (P == 1 && Q.n_groups > 1 && S.n_long == 0) {
    int big = 0, small = 1 << 30;
    for (int i = 0; i < Q.n_groups; ++i) {
      big = std::max(big, Q.group[8 * (size_t)i + 4]);
      small = std::min(small, Q.group[8 * (size_t)i + 4]);
    }
    const int ng = (int)(((int64_t)no + target - 1) / target);
    if (tail == 0 && Q.n_groups == ng)
      CHECK(big - small <= 2 * S.max_track, "groups unbalanced: %d vs %d", big, small);
    CHECK(big <= target + S.max_track, "a group of %d observations for a target of %d", big, target);
  }
  // camera-major rows of the group slots
  CHECK(Q.cam_ptr[0] == 0 && Q.cam_ptr[nc] == Q.n_gslots, "series rows do not cover the group slots");
  {
    std::vector<char> seen_row(Q.n_gslots, 0);
    std::vector<int> row_group(Q.n_gslots, -1);
    for (int s = 0; s < Q.n_gslots; ++s) {
      const int r = Q.gslot_row[s], cam = Q.gslot_cam[s];
      CHECK(r >= 0 && r < Q.n_gslots && !seen_row[r], "gslot_row is not a permutation at %d", s);
      seen_row[r] = 1;
      CHECK(r >= Q.cam_ptr[cam] && r < Q.cam_ptr[cam + 1], "group slot %d's row is not its camera's", s);
      // landmark order: the group's first chunk (a long group's slot: its chunk)
      row_group[r] = slot_key[s];
    }
    for (int cam = 0; cam < nc; ++cam)
      for (int r = Q.cam_ptr[cam] + 1; r < Q.cam_ptr[cam + 1]; ++r)
        CHECK(row_group[r] > row_group[r - 1], "camera %d's rows are not in landmark order", cam);
  }

  // camera rounds for a grid of G blocks over the series rows
  CamSchedule cs;
  build_cam_schedule(Q.cam_ptr, nc, &cs);
  for (int c = 0; c < nc; ++c) {
    const int r0 = Q.cam_ptr[c], r1 = Q.cam_ptr[c + 1];
    const int i0 = cs.cam_item[c], i1 = cs.cam_item[c + 1];
    CHECK(i1 - i0 == cam_chunks(r1 - r0) && i1 - i0 <= kRoundItems, "camera %d's chunk count", c);
    int q = r0;
    for (int i = i0; i < i1; ++i) {
      CHECK(cs.item_q[2 * i] == q && cs.item_q[2 * i + 1] >= q &&
                cs.item_q[2 * i + 1] - q <= cam_chunk_rows(r1 - r0),
            "camera %d's chunks do not tile its rows", c);
      q = cs.item_q[2 * i + 1];
    }
    CHECK(q == r1, "camera %d's chunks end at %d, not %d", c, q, r1);
  }
  CamRoundList rl;
  build_cam_rounds(cs, nc, G, &rl);
  const int R = (int)rl.round_cam.size() - 1;
  CHECK(rl.round_cam.front() == 0 && rl.round_cam.back() == nc, "rounds do not cover the cameras");
  for (int r = 0; r < R; ++r) {
    const int c0 = rl.round_cam[r], c1 = rl.round_cam[r + 1];
    CHECK(c1 > c0, "round %d is empty", r);
    CHECK(rl.round_item[r] == cs.cam_item[c0] && rl.round_item[r + 1] == cs.cam_item[c1],
          "round %d's items are not its cameras'", r);
    CHECK(c1 - c0 <= kRoundItems && rl.round_item[r + 1] - rl.round_item[r] <= kRoundItems,
          "round %d holds %d cameras and %d items", r, c1 - c0,
          rl.round_item[r + 1] - rl.round_item[r]);
  }
  CHECK((int)rl.block_round.size() == G + 1 && rl.block_round[0] == 0 && rl.block_round[G] == R,
        "block_round does not split the rounds over the grid");
  for (int b = 0; b < G; ++b)
    CHECK(rl.block_round[b + 1] >= rl.block_round[b], "block_round decreases at %d", b);

  std::printf("ok wide=%d tiles=%d slots=%d rounds=%d groups=%d chunks=%d gslots=%d\n", n_wide,
              S.n_tiles,
              S.n_slots, R, Q.n_groups, Q.n_chunks, Q.n_gslots);
  return 0;
}
