"""Seeded synthetic bundle-adjustment problems in the BAL camera model.

This module only draws random numbers and lays them out; it computes no residual, Jacobian,
normal-equation block or solve.  Both the FP64 CPU oracle (``oracle/``) and the CUDA path
(``paper_2204_12834_gb300``) read the problems it makes, and neither shares any other code.

The one piece of geometry here is the forward camera model used to *synthesise* pixel
observations from the ground truth (obs = projection(gt) + pixel noise) and to reject
landmark/camera pairs that would put the point behind the camera.  It is written with the
rotation *matrix* form of Rodrigues' formula, unlike both solvers, and it only shapes the data:
a mistake here changes which problem is solved, never whether the two solvers agree.

Camera vector (BAL convention, 9 parameters, Sec. 4 with d_p = 9):
    [w0, w1, w2, t0, t1, t2, f, k1, k2]
with angle-axis rotation w, translation t, focal length f and radial distortion k1, k2.

Problem recipe (stand-ins for the BAL suite, whose files are not available):
  * cameras: w ~ N(0, 0.1^2) per component, t ~ N(0, 1), f = 500, k1, k2 ~ N(0, 1e-3^2)
  * landmarks: uniform in the box [-5, 5] x [-5, 5] x [-15, -5]; a landmark whose point lands
    at camera depth P_z > -1 for any observing camera is redrawn
  * observations: projection of the ground truth plus N(0, 1 px^2) per coordinate
  * initial state (Appendix B noise (m, sigma) = (0, 0.01)): additive N(0, sigma^2) on the
    landmark coordinates and on camera w and t; f scaled by (1 + sigma N(0, 1)); k1, k2 kept
  * visibility: "uniform" (k distinct random cameras), "clustered" (k distinct cameras in a
    window [c, c + width) mod n_c around a random centre c), track length k drawn per landmark
  * observation order is shuffled so that consumers must sort
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

__all__ = ["Problem", "make_problem", "PRESETS", "preset", "make_batch"]


@dataclasses.dataclass
class Problem:
    """One BA problem: ground truth, initial state and observations (all float64 / int32)."""

    name: str
    cams_gt: np.ndarray      # [n_c, 9]
    lms_gt: np.ndarray       # [n_l, 3]
    cams0: np.ndarray        # [n_c, 9] initial (perturbed) cameras
    lms0: np.ndarray         # [n_l, 3] initial (perturbed) landmarks
    obs: np.ndarray          # [n_o, 2] pixel observations
    cam_idx: np.ndarray      # [n_o] int32
    lm_idx: np.ndarray       # [n_o] int32
    weights: Optional[np.ndarray]  # [n_o] or None (all ones)
    noise: np.ndarray        # [n_o, 2] the pixel noise that was added to the exact projection

    @property
    def n_cams(self) -> int:
        return int(self.cams0.shape[0])

    @property
    def n_lms(self) -> int:
        return int(self.lms0.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs.shape[0])


def _rot_matrices(w: np.ndarray) -> np.ndarray:
    """Rotation matrices exp([w]x) for angle-axis rows w [n, 3] (matrix form of Rodrigues)."""
    theta = np.linalg.norm(w, axis=1)
    safe = np.where(theta > 0, theta, 1.0)
    k = w / safe[:, None]
    K = np.zeros((w.shape[0], 3, 3))
    K[:, 0, 1], K[:, 0, 2] = -k[:, 2], k[:, 1]
    K[:, 1, 0], K[:, 1, 2] = k[:, 2], -k[:, 0]
    K[:, 2, 0], K[:, 2, 1] = -k[:, 1], k[:, 0]
    s, c = np.sin(theta)[:, None, None], np.cos(theta)[:, None, None]
    R = np.eye(3)[None] + s * K + (1.0 - c) * (K @ K)
    return R


def _camera_points(cams: np.ndarray, lms: np.ndarray, cam_idx: np.ndarray, lm_idx: np.ndarray) -> np.ndarray:
    R = _rot_matrices(cams[:, 0:3])
    return np.einsum("oij,oj->oi", R[cam_idx], lms[lm_idx]) + cams[cam_idx, 3:6]


def _synth_pixels(cams, lms, cam_idx, lm_idx):
    P = _camera_points(cams, lms, cam_idx, lm_idx)
    p = -P[:, 0:2] / P[:, 2:3]
    n2 = (p * p).sum(1)
    c = cams[cam_idx]
    scale = c[:, 6] * (1.0 + c[:, 7] * n2 + c[:, 8] * n2 * n2)
    return scale[:, None] * p


def _distinct_offsets(rng: np.random.Generator, k: np.ndarray, width: np.ndarray) -> list:
    """For each landmark pick k[i] distinct offsets in [0, width[i]) (chunked argsort of keys)."""
    out = [None] * len(k)
    for w in np.unique(width):
        sel = np.nonzero(width == w)[0]
        for s in range(0, len(sel), 65536):
            chunk = sel[s:s + 65536]
            keys = rng.random((len(chunk), int(w)))
            order = np.argsort(keys, axis=1)
            for j, i in enumerate(chunk):
                out[i] = order[j, : k[i]]
    return out


def _track_lengths(rng, n_l, spec):
    kind = spec[0]
    if kind == "uniform":
        lo, hi = spec[1], spec[2]
        return rng.integers(lo, hi + 1, size=n_l)
    if kind == "powerlaw":
        alpha, lo, hi = spec[1], spec[2], spec[3]
        ks = np.arange(lo, hi + 1)
        p = ks.astype(np.float64) ** (-alpha)
        p /= p.sum()
        return rng.choice(ks, size=n_l, p=p)
    if kind == "long":
        # ("long", kmin, kmax, (k_0, k_1, ...)): landmarks 0, 1, ... get the listed track
        # lengths (long tracks), the others U{kmin..kmax}
        lo, hi, long = spec[1], spec[2], np.asarray(spec[3], dtype=np.int64)
        k = rng.integers(lo, hi + 1, size=n_l)
        k[:long.size] = long[:n_l]
        return k
    raise ValueError(f"unknown track-length spec {spec}")


def make_problem(n_cams: int, n_lms: int, track=("uniform", 2, 6), visibility="uniform",
                 window=8, seed: int = 0, sigma_init: float = 0.01, pixel_noise: float = 1.0,
                 weighted: bool = False, name: str = "custom", shuffle: bool = True) -> Problem:
    """Draw one problem.

    track: ("uniform", kmin, kmax) or ("powerlaw", alpha, kmin, kmax) track-length law, or
    ("long", kmin, kmax, lengths): the first landmarks get the listed lengths, the rest uniform.
    visibility: "uniform" (k distinct cameras out of all) or "clustered" (k distinct cameras in
    [c, c + width) mod n_cams, width = max(window, 2 k) for power-law tracks, else window).
    """
    rng = np.random.default_rng(seed)
    n_c, n_l = int(n_cams), int(n_lms)
    cams = np.zeros((n_c, 9))
    cams[:, 0:3] = rng.normal(0.0, 0.1, size=(n_c, 3))
    cams[:, 3:6] = rng.normal(0.0, 1.0, size=(n_c, 3))
    cams[:, 6] = 500.0
    cams[:, 7:9] = rng.normal(0.0, 1e-3, size=(n_c, 2))

    k = _track_lengths(rng, n_l, track)
    k = np.minimum(k, n_c)
    if visibility == "uniform":
        width = np.full(n_l, n_c)
        centre = np.zeros(n_l, dtype=np.int64)
    elif visibility == "clustered":
        if track[0] == "powerlaw":
            width = np.minimum(np.maximum(2 * k, window), n_c)
        else:
            width = np.minimum(np.maximum(k, window), n_c)
        centre = rng.integers(0, n_c, size=n_l)
    else:
        raise ValueError(visibility)
    offs = _distinct_offsets(rng, k, width)
    lm_idx = np.repeat(np.arange(n_l, dtype=np.int64), k)
    cam_idx = np.concatenate([(centre[i] + offs[i]) % n_c for i in range(n_l)]).astype(np.int64)

    lo = np.array([-5.0, -5.0, -15.0])
    hi = np.array([5.0, 5.0, -5.0])
    lms = lo + (hi - lo) * rng.random((n_l, 3))
    for _ in range(100):
        Pz = _camera_points(cams, lms, cam_idx, lm_idx)[:, 2]
        bad = np.unique(lm_idx[Pz > -1.0])
        if bad.size == 0:
            break
        lms[bad] = lo + (hi - lo) * rng.random((bad.size, 3))
    else:
        raise RuntimeError("could not place landmarks in front of their cameras")

    noise = rng.normal(0.0, pixel_noise, size=(lm_idx.size, 2))
    obs = _synth_pixels(cams, lms, cam_idx, lm_idx) + noise

    cams0 = cams.copy()
    cams0[:, 0:6] += rng.normal(0.0, sigma_init, size=(n_c, 6))
    cams0[:, 6] *= 1.0 + sigma_init * rng.normal(0.0, 1.0, size=n_c)
    lms0 = lms + rng.normal(0.0, sigma_init, size=(n_l, 3))
    weights = rng.uniform(0.5, 1.5, size=lm_idx.size) if weighted else None

    if shuffle:
        perm = rng.permutation(lm_idx.size)
        obs, noise, cam_idx, lm_idx = obs[perm], noise[perm], cam_idx[perm], lm_idx[perm]
        if weights is not None:
            weights = weights[perm]
    return Problem(name=name, cams_gt=cams, lms_gt=lms, cams0=cams0, lms0=lms0,
                   obs=np.ascontiguousarray(obs), cam_idx=cam_idx.astype(np.int32),
                   lm_idx=lm_idx.astype(np.int32), weights=weights, noise=noise)


# Named workloads (sizes in the name).  Seeds are fixed per workload.
PRESETS = {
    # parity case: 16 cameras, 1,000 landmarks, tracks U{2..6}, uniform visibility (~4,000 obs)
    "uniform_16c_1000l": dict(n_cams=16, n_lms=1000, track=("uniform", 2, 6),
                              visibility="uniform", seed=1001),
    # Ladybug-1197-sized: 1,200 cameras, 160,000 landmarks, tracks U{3,4}, clustered (~560k obs)
    "clustered_1200c_160000l": dict(n_cams=1200, n_lms=160000, track=("uniform", 3, 4),
                                    visibility="clustered", window=8, seed=1002),
    # 3,000 cameras, 400,000 landmarks, tracks U{3,4}, clustered (~1.4M obs): Jacobians larger
    # than the GPU's L2, for profiling the series kernels
    "clustered_3000c_400000l": dict(n_cams=3000, n_lms=400000, track=("uniform", 3, 4),
                                    visibility="clustered", window=8, seed=1006),
    # Venice-1778-sized: 10,000 cameras, 1,000,000 landmarks, power-law tracks on [2, 50] (~5M obs)
    "powerlaw_10000c_1000000l": dict(n_cams=10000, n_lms=1000000,
                                     track=("powerlaw", 2.14, 2, 50), visibility="clustered",
                                     window=64, seed=1003),
    # weighted problem: 200 cameras, 20,000 landmarks, tracks U{2..6}, weights U(0.5, 1.5)
    "weighted_200c_20000l": dict(n_cams=200, n_lms=20000, track=("uniform", 2, 6),
                                 visibility="uniform", weighted=True, seed=1005),
}


def preset(name: str, **overrides) -> Problem:
    kw = dict(PRESETS[name])
    kw.update(overrides)
    return make_problem(name=name, **kw)


def make_batch(n_problems: int = 256, seed: int = 1004, cams=(8, 200), lms=(500, 20000),
               track=(2, 8)):
    """Independent problems of uneven sizes (clustered visibility, window 8)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        nc = int(rng.integers(cams[0], cams[1] + 1))
        nl = int(rng.integers(lms[0], lms[1] + 1))
        out.append(make_problem(nc, nl, track=("uniform", track[0], track[1]),
                                visibility="clustered", window=8,
                                seed=int(rng.integers(0, 2**31 - 1)), name=f"batch{i}"))
    return out
