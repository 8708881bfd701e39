"""The seeded generator behind every workload, checked against the input recipe it implements:
BAL-model cameras (angle-axis omega ~ N(0, 0.1^2), t ~ N(0, 1), f = 500, k1, k2 ~ N(0, 1e-3^2)),
landmarks uniform in [-5, 5]^2 x [-15, -5] and at depth <= -1 in every observing camera (the
BAL camera looks along -z), 1 px Gaussian pixel noise, the initial state perturbed by 1 %
(omega, t and landmarks additively, f multiplicatively, k1 and k2 untouched), distinct cameras
per track, clustered visibility inside a window of cameras, uniform or power-law track lengths,
and the named workloads' sizes.  The depth test uses the oracle's Rodrigues rotation, written
independently of the generator's matrix form."""
import numpy as np
import pytest

import bal_synth
from oracle import camera_model as cm


@pytest.fixture(scope="module")
def medium():
    return bal_synth.make_problem(2000, 20000, track=("uniform", 2, 6), visibility="clustered",
                                  window=8, seed=31)


def test_seeded_and_deterministic():
    a = bal_synth.make_problem(50, 400, seed=5)
    b = bal_synth.make_problem(50, 400, seed=5)
    c = bal_synth.make_problem(50, 400, seed=6)
    for f in ("cams0", "lms0", "obs", "cam_idx", "lm_idx", "cams_gt", "lms_gt"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert not np.array_equal(a.obs, c.obs)


def test_camera_and_landmark_distributions(medium):
    g = medium.cams_gt
    assert abs(g[:, 0:3].std() - 0.1) < 0.005 and abs(g[:, 0:3].mean()) < 0.005
    assert abs(g[:, 3:6].std() - 1.0) < 0.05
    assert np.all(g[:, 6] == 500.0)
    assert abs(g[:, 7:9].std() - 1e-3) < 1e-4
    X = medium.lms_gt
    assert np.all(X[:, 0:2] >= -5) and np.all(X[:, 0:2] <= 5)
    assert np.all(X[:, 2] >= -15) and np.all(X[:, 2] <= -5)


def test_landmarks_in_front_of_every_observing_camera(medium):
    p = medium
    cam, X = p.cams_gt[p.cam_idx], p.lms_gt[p.lm_idx]
    RX = cm.rotate([cam[:, 0], cam[:, 1], cam[:, 2]], [X[:, 0], X[:, 1], X[:, 2]])
    Pz = RX[2] + cam[:, 5]
    assert np.all(Pz <= -1.0)


def test_pixel_noise_and_initial_perturbation(medium):
    p = medium
    assert abs(p.noise.mean()) < 0.01 and abs(p.noise.std() - 1.0) < 0.01
    d = p.cams0 - p.cams_gt
    assert abs(d[:, 0:6].std() - 0.01) < 0.0005
    assert abs((p.cams0[:, 6] / p.cams_gt[:, 6] - 1.0).std() - 0.01) < 0.001
    assert np.array_equal(p.cams0[:, 7:9], p.cams_gt[:, 7:9])
    assert abs((p.lms0 - p.lms_gt).std() - 0.01) < 0.0002


def covering_arc(cams, n_c):
    """Length of the shortest arc of the camera ring (mod n_c) that holds every camera."""
    a = np.sort(cams)
    gaps = np.diff(np.concatenate([a, [a[0] + n_c]]))
    return n_c - gaps.max() + 1


def test_tracks_distinct_and_clustered(medium):
    p = medium
    order = np.argsort(p.lm_idx, kind="stable")
    seg = np.concatenate([[0], np.cumsum(np.bincount(p.lm_idx, minlength=p.n_lms))])
    cams = p.cam_idx[order]
    k = np.diff(seg)
    assert k.min() == 2 and k.max() == 6 and abs(k.mean() - 4.0) < 0.05
    for l in range(0, p.n_lms, 37):
        c = cams[seg[l]:seg[l + 1]]
        assert len(np.unique(c)) == len(c)
        assert covering_arc(c, p.n_cams) <= 8
    # the observations are shuffled, not grouped by landmark or camera
    assert np.any(np.diff(p.lm_idx) < 0) and np.any(np.diff(p.cam_idx) < 0)


def test_powerlaw_tracks_and_their_window():
    """p(k) proportional to k^-2.14 on [2, 50], each track inside a window of max(2k, 64)."""
    p = bal_synth.preset("powerlaw_10000c_1000000l")
    assert (p.n_cams, p.n_lms, p.n_obs) == (10000, 1000000, 5000570)
    k = np.bincount(p.lm_idx, minlength=p.n_lms)
    assert k.min() == 2 and k.max() == 50
    ks = np.arange(2, 51)
    pk = ks ** -2.14
    pk /= pk.sum()
    sd = np.sqrt((ks ** 2 * pk).sum() - (ks * pk).sum() ** 2)
    assert abs(k.mean() - (ks * pk).sum()) < 5 * sd / np.sqrt(p.n_lms)
    counts = np.bincount(k, minlength=51)
    assert abs(counts[2] / counts[3] - 1.5 ** 2.14) < 0.04
    order = np.argsort(p.lm_idx, kind="stable")
    seg = np.concatenate([[0], np.cumsum(k)])
    cams = p.cam_idx[order]
    for l in range(0, p.n_lms, 997):
        c = cams[seg[l]:seg[l + 1]]
        assert len(np.unique(c)) == len(c)
        assert covering_arc(c, p.n_cams) <= max(2 * len(c), 64)


@pytest.mark.parametrize("name,sizes", [
    ("uniform_16c_1000l", (16, 1000, None)),
    ("clustered_1200c_160000l", (1200, 160000, 559912)),
    ("weighted_200c_20000l", (200, 20000, None)),
])
def test_named_workload_sizes(name, sizes):
    p = bal_synth.preset(name)
    assert (p.n_cams, p.n_lms) == sizes[:2]
    if sizes[2] is not None:
        assert p.n_obs == sizes[2]
    if name.startswith("weighted"):
        assert p.weights.min() >= 0.5 and p.weights.max() <= 1.5
        assert abs(p.weights.mean() - 1.0) < 0.01
    else:
        assert p.weights is None


def test_batch_of_uneven_problems():
    ps = bal_synth.make_batch(256)
    assert len(ps) == 256
    assert sum(q.n_cams for q in ps) == 28099
    assert sum(q.n_lms for q in ps) == 2532769
    assert sum(q.n_obs for q in ps) == 12664995
    for q in ps[:16]:
        assert 8 <= q.n_cams <= 200 and 500 <= q.n_lms <= 20000
        k = np.bincount(q.lm_idx, minlength=q.n_lms)
        assert k.min() >= 2 and k.max() <= 8
