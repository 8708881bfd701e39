"""Host-side helpers of bench.py that the reported figures rest on, checked against plainly
written brute-force counts on small problems: the explicit block-sparse S footprint (camera
pairs that share a landmark) and the slot count of the tile packing (landmarks ordered by their
smallest observing camera, whole tracks, at most 256 observations, 256 landmarks and 128
distinct cameras per tile)."""
import itertools

import numpy as np
import pytest

import bal_synth
import bench


def brute_pairs(p):
    pairs = set()
    for l in range(p.n_lms):
        cams = sorted(set(p.cam_idx[p.lm_idx == l].tolist()))
        for a, b in itertools.combinations_with_replacement(cams, 2):
            pairs.add((a, b))
    return len(pairs)


def brute_slots(p, tile_obs=256, tile_lms=256, tile_cams=128):
    first = {l: min(p.cam_idx[p.lm_idx == l].tolist()) for l in range(p.n_lms)
             if np.any(p.lm_idx == l)}
    order = sorted(range(p.n_lms), key=lambda l: (first.get(l, p.n_cams), l))
    tiles, cur, obs = [], [], 0
    cams = set()
    for l in order:
        track = p.cam_idx[p.lm_idx == l].tolist()
        fits = (obs + len(track) <= tile_obs and len(cur) + 1 <= tile_lms
                and len(cams | set(track)) <= tile_cams)
        if cur and not fits:
            tiles.append(cams)
            cur, obs, cams = [], 0, set()
        cur.append(l)
        obs += len(track)
        cams |= set(track)
    tiles.append(cams)
    return sum(len(t) for t in tiles)


CASES = [
    dict(n_cams=12, n_lms=150, track=("uniform", 2, 6), seed=71),
    dict(n_cams=40, n_lms=300, track=("powerlaw", 2.14, 2, 30), visibility="clustered", seed=72),
    dict(n_cams=200, n_lms=120, track=("uniform", 40, 60), seed=73),  # tiles capped by cameras
]


@pytest.mark.parametrize("kw", CASES)
def test_explicit_s_bytes_counts_camera_pairs(kw):
    p = bal_synth.make_problem(**kw)
    assert bench.explicit_s_bytes(p) == brute_pairs(p) * 81 * 8


@pytest.mark.parametrize("kw", CASES)
def test_schedule_slots_matches_a_plain_packing(kw):
    p = bal_synth.make_problem(**kw)
    assert bench.schedule_slots(p) == brute_slots(p)


def test_small_tiles_change_the_slot_count():
    """The caps matter: smaller tiles can only add slots (a camera split over more tiles)."""
    p = bal_synth.make_problem(n_cams=30, n_lms=400, track=("uniform", 2, 6),
                               visibility="clustered", seed=74)
    assert bench.schedule_slots(p, tile_obs=64) >= bench.schedule_slots(p)
    assert bench.schedule_slots(p, tile_obs=64) == brute_slots(p, tile_obs=64)


def test_minimal_series_units_per_observation():
    """Per observation the minimal term moves 24 s + 4 bytes and does 48 FMA (96 flops)."""
    p = bal_synth.make_problem(n_cams=10, n_lms=100, track=("uniform", 2, 4), seed=75)
    b8, f = bench.series_term_units(p, 8)
    b4, _ = bench.series_term_units(p, 4)
    assert b8 - b4 == p.n_obs * 24 * 4 + p.n_lms * 6 * 4
    assert f == 96 * p.n_obs + 18 * p.n_lms + 162 * p.n_cams


def test_step_stats():
    s = bench.step_stats([3.0, 1.0, 2.0, 10.0, 2.0])
    assert s["median"] == 2.0 and s["n"] == 5 and s["p10"] <= s["median"] <= s["p90"] <= 10.0
    assert bench.step_stats([])["median"] is None
