"""The library's tile schedule (schedule.cpp), built on the host without a GPU and checked by
tests/cpp/schedule_check.cpp against the properties the kernels rely on: observations sorted by
(landmark, camera); tiles of whole landmarks of one problem within the observation, landmark
and camera caps; slots equal to each tile's cameras in ascending order, with positions that
sort the tile by camera; camera-major rows in tile order; camera chunks that tile each
camera's rows; rounds of at most 28 cameras and items split over the grid; series groups within
each precision's camera cap (256 FP32 bulk, 96 FP64), landmarks wider than the cap and long
tracks' pieces in groups of their own."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import bal_synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2204_12834_gb300", "csrc")


def cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("sched") / "schedule_check")
    cmd = [cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc,
           os.path.join(ROOT, "tests", "cpp", "schedule_check.cpp"),
           os.path.join(CSRC, "schedule.cpp"), "-o", exe]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-2000:]
    return exe


def run(checker, tmp_path, problems, grid=456):
    cam_off = np.cumsum([0] + [q.n_cams for q in problems]).astype(np.int32)
    lm_off = np.cumsum([0] + [q.n_lms for q in problems]).astype(np.int32)
    cam = np.concatenate([q.cam_idx + cam_off[i] for i, q in enumerate(problems)]).astype(np.int32)
    lm = np.concatenate([q.lm_idx + lm_off[i] for i, q in enumerate(problems)]).astype(np.int32)
    hdr = np.array([len(problems), cam_off[-1], lm_off[-1], len(cam), grid], dtype=np.int32)
    path = tmp_path / "problem.bin"
    with open(path, "wb") as f:
        for a in (hdr, cam_off, lm_off, cam, lm):
            f.write(np.ascontiguousarray(a, dtype="<i4").tobytes())
    out = subprocess.run([checker, str(path)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
    return out.stdout


CASES = {
    "uniform": lambda: bal_synth.make_problem(16, 1000, track=("uniform", 2, 6), seed=81),
    "clustered": lambda: bal_synth.make_problem(300, 20000, track=("uniform", 3, 4),
                                                visibility="clustered", seed=82),
    "powerlaw": lambda: bal_synth.make_problem(200, 6000, track=("powerlaw", 2.14, 2, 50),
                                               visibility="clustered", seed=83),
    "wide_tracks": lambda: bal_synth.make_problem(300, 200, track=("uniform", 40, 60), seed=84),
    "tiny": lambda: bal_synth.make_problem(3, 7, track=("uniform", 2, 3), seed=85),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_schedule_properties(checker, tmp_path, name):
    """... and bench.py's mirror of the packer (the slot count behind its design bytes)
    counts the library's slots."""
    import bench
    p = CASES[name]()
    out = run(checker, tmp_path, [p])
    slots = int(out.split("slots=")[1].split()[0])
    assert bench.schedule_slots(p) == slots


def test_schedule_with_a_256_camera_track(checker, tmp_path):
    """One landmark seen by 256 distinct cameras takes a tile of its own (256 slots)."""
    p = bal_synth.make_problem(256, 300, track=("uniform", 2, 6), seed=86)
    extra = np.setdiff1d(np.arange(256), p.cam_idx[p.lm_idx == 0])
    p.cam_idx = np.concatenate([p.cam_idx, extra]).astype(p.cam_idx.dtype)
    p.lm_idx = np.concatenate([p.lm_idx, np.zeros(len(extra), dtype=p.lm_idx.dtype)])
    assert np.sum(p.lm_idx == 0) == 256
    run(checker, tmp_path, [p])


def test_schedule_with_landmarks_wider_than_the_fp64_cap(checker, tmp_path):
    """FP64 groups hold at most 96 cameras (odd grids make the checker use that cap): landmarks
    seen by 256, 150 and 97 cameras each become a group of their own (one chunk with its own
    slots), one seen by exactly 96 does not; under the FP32-bulk cap of 256 none does."""
    p = bal_synth.make_problem(256, 300, track=("uniform", 2, 6), seed=93)
    for lm, k in ((0, 256), (1, 150), (2, 97), (3, 96)):
        seen = p.cam_idx[p.lm_idx == lm]
        extra = np.setdiff1d(np.arange(k), seen)[:k - len(np.unique(seen))]
        p.cam_idx = np.concatenate([p.cam_idx, extra]).astype(p.cam_idx.dtype)
        p.lm_idx = np.concatenate([p.lm_idx, np.full(len(extra), lm, dtype=p.lm_idx.dtype)])
        assert len(np.unique(p.cam_idx[p.lm_idx == lm])) == max(k, len(np.unique(seen)))
    assert run(checker, tmp_path, [p], grid=455).startswith("ok wide=3 ")
    assert run(checker, tmp_path, [p], grid=456).startswith("ok wide=0 ")


def test_schedule_with_a_repeated_observation(checker, tmp_path):
    """A (camera, landmark) pair observed twice is two rows of the same slot."""
    p = bal_synth.make_problem(10, 50, track=("uniform", 2, 4), seed=88)
    p.cam_idx = np.concatenate([p.cam_idx, p.cam_idx[:1]])
    p.lm_idx = np.concatenate([p.lm_idx, p.lm_idx[:1]])
    run(checker, tmp_path, [p])


def test_batch_schedule_properties(checker, tmp_path):
    """A batch of uneven problems: no tile holds two problems; the same checks per tile."""
    rng = np.random.default_rng(87)
    problems = [bal_synth.make_problem(int(rng.integers(8, 60)), int(rng.integers(50, 1500)),
                                       track=("uniform", 2, 8), visibility="clustered",
                                       seed=int(rng.integers(1 << 30))) for _ in range(8)]
    run(checker, tmp_path, problems, grid=152)


@pytest.mark.parametrize("workload", ["clustered_1200c_160000l", "powerlaw_10000c_1000000l"])
def test_full_size_schedules(checker, tmp_path, workload):
    """The two full-size single problems the benchmark times, at the grids of the persistent
    kernel (3 and 4 blocks per SM on 152 SMs); bench.py's slot mirror counts the same slots."""
    import bench
    p = bal_synth.preset(workload)
    for grid in (456, 608):
        out = run(checker, tmp_path, [p], grid=grid)
        slots = int(out.split("slots=")[1].split()[0])
    assert bench.schedule_slots(p) == slots


@pytest.mark.parametrize("lengths", [(257,), (300, 700, 2000), (512, 513, 256, 1024)])
def test_schedule_with_long_tracks(checker, tmp_path, lengths):
    """Tracks of more than 256 observations: split into near-equal pieces of at most 256 (in
    camera order), each alone in its tile, the pieces of a track forming one series group of
    one chunk per piece; the other landmarks are scheduled as usual."""
    p = bal_synth.make_problem(2100, 3000, track=("long", 2, 6, lengths), seed=89)
    assert sorted(np.bincount(p.lm_idx)[:len(lengths)]) == sorted(lengths)
    for grid in (456, 40):
        out = run(checker, tmp_path, [p], grid=grid)
        assert out.startswith("ok")


def test_batch_schedule_with_long_tracks(checker, tmp_path):
    """A batch whose problems hold long tracks (and one that holds none)."""
    problems = [bal_synth.make_problem(600, 400, track=("long", 2, 5, (300,)), seed=90),
                bal_synth.make_problem(40, 300, track=("uniform", 2, 5), seed=91),
                bal_synth.make_problem(900, 200, track=("long", 2, 5, (800, 260)), seed=92)]
    run(checker, tmp_path, problems, grid=152)
