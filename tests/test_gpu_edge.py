"""GPU edge cases against the oracle: no observations, unobserved cameras and landmarks, the
longest supported track (256 observations of one landmark), tiles with 256 distinct cameras,
a single camera, m = 0, device-resident inputs, non-SPD damping and non-finite states."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import OracleRef, check_step_blocks, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def poba():
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    return m


def check_series(poba, p, lam=1e-3, m=6, tol=1e-10, precision=0):
    ref = OracleRef(p)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights,
                       precision=precision, options=poba.ba_default_options(eps=0.0, max_inner=m))
    poba.ba_linearize(h)
    poba.ba_solve_schur_power(h, lam)
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(lam, 0.0, m)
    assert rel(dxp, o["x"]) < tol
    assert rel(dxl, o["xl"]) < tol
    check_step_blocks(dxp, dxl, o["x"], o["xl"], precision)
    return h


def test_unobserved_cameras_and_landmarks(poba):
    p = bal_synth.make_problem(12, 500, seed=101)
    # append a camera and two landmarks that nothing observes
    p.cams0 = np.vstack([p.cams0, p.cams0[:1] + 0.1])
    p.lms0 = np.vstack([p.lms0, p.lms0[:2] + 0.5])
    check_series(poba, p)


def test_longest_track_and_wide_tiles(poba):
    rng = np.random.default_rng(5)
    p = bal_synth.make_problem(256, 400, track=("uniform", 2, 6), seed=103)
    # landmark 0 observed 256 times (every camera once)
    extra = 256 - int(np.sum(p.lm_idx == 0))
    cams_missing = np.setdiff1d(np.arange(256), p.cam_idx[p.lm_idx == 0])[:extra]
    from oracle import camera_model as cm
    add_c = cams_missing.astype(np.int32)
    add_l = np.zeros(len(add_c), np.int32)
    pix = np.stack(cm.project([p.cams_gt[add_c, j] for j in range(9)],
                              [p.lms_gt[add_l, j] for j in range(3)]), 1)
    p.obs = np.vstack([p.obs, pix + rng.normal(0, 1, pix.shape)])
    p.cam_idx = np.concatenate([p.cam_idx, add_c])
    p.lm_idx = np.concatenate([p.lm_idx, add_l])
    assert np.sum(p.lm_idx == 0) == 256
    check_series(poba, p)
    # FP32-bulk: a 256-observation chunk with 256 distinct cameras (every lane of every warp in
    # one landmark segment); the persistent kernel and the per-term launches agree bit for bit
    h32 = check_series(poba, p, tol=1e-4, precision=1)
    steps = []
    for mode in (1, 2, 3, 4, 5):
        h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=1,
                           options=poba.ba_default_options(eps=0.0, max_inner=6, series_exec=mode))
        poba.ba_linearize(h)
        poba.ba_solve_schur_power(h, 1e-3)
        steps.append(poba.ba_get_step(h))
    for st in steps[1:]:
        assert np.array_equal(st[0], steps[0][0]) and np.array_equal(st[1], steps[0][1])


def test_landmarks_wider_than_the_fp64_group(poba):
    """FP64 groups hold at most 96 cameras: landmarks seen by 150 and 97 cameras run as groups
    of their own (the long-group body), one seen by 96 cameras in an ordinary group. FP64 series
    against the oracle at fixed m and with the stop rule; every form gives the same bits (forms
    4 and 5 fall back to 3 on such a problem, and ba_set_schedule refuses them)."""
    rng = np.random.default_rng(6)
    p = bal_synth.make_problem(200, 600, track=("uniform", 2, 6), seed=113)
    from oracle import camera_model as cm
    for lm, k in ((0, 150), (1, 97), (2, 96)):
        seen = p.cam_idx[p.lm_idx == lm]
        add_c = np.setdiff1d(np.arange(k), seen)[:k - len(np.unique(seen))].astype(np.int32)
        add_l = np.full(len(add_c), lm, np.int32)
        pix = np.stack(cm.project([p.cams_gt[add_c, j] for j in range(9)],
                                  [p.lms_gt[add_l, j] for j in range(3)]), 1)
        p.obs = np.vstack([p.obs, pix + rng.normal(0, 1, pix.shape)])
        p.cam_idx = np.concatenate([p.cam_idx, add_c])
        p.lm_idx = np.concatenate([p.lm_idx, add_l])
    check_series(poba, p)
    check_series(poba, p, lam=1e-2, m=20)
    steps = []
    for mode in (0, 1, 2, 3, 4, 5):
        h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=0,
                           options=poba.ba_default_options(eps=0.01, max_inner=12,
                                                           series_exec=mode))
        poba.ba_linearize(h)
        info = poba.ba_solve_schur_power(h, 1e-3)
        steps.append((info["inner_iters"], poba.ba_get_step(h)))
    for st in steps[1:]:
        assert st[0] == steps[0][0]
        assert np.array_equal(st[1][0], steps[0][1][0]) and np.array_equal(st[1][1], steps[0][1][1])
    with pytest.raises(poba.PobaError):
        poba.ba_set_schedule(h, series_exec=5, blocks_per_sm=1)


def test_no_observations(poba):
    p = bal_synth.make_problem(3, 10, seed=105)
    h = poba.ba_create(p.cams0, p.lms0, p.obs[:0], p.cam_idx[:0], p.lm_idx[:0],
                       options=poba.ba_default_options(max_inner=4))
    assert poba.ba_cost(h) == 0.0
    assert poba.ba_linearize(h) == 0.0
    info = poba.ba_solve_schur_power(h, 1e-3)
    dxp, dxl = poba.ba_get_step(h)
    assert info["inner_iters"] == 0 and info["stopped"] == 1
    assert np.all(dxp == 0) and np.all(dxl == 0)


def test_single_camera_single_landmark(poba):
    p = bal_synth.make_problem(1, 1, track=("uniform", 1, 1), seed=107)
    check_series(poba, p, lam=1e-2, m=3)


def test_zero_terms(poba):
    p = bal_synth.make_problem(8, 200, seed=109)
    check_series(poba, p, lam=1e-2, m=0)


def test_device_inputs_and_stream(poba):
    import torch
    p = bal_synth.make_problem(16, 600, seed=111)
    s = torch.cuda.Stream()
    dev = lambda a: torch.as_tensor(a).cuda()
    with torch.cuda.stream(s):
        h = poba.ba_create(dev(p.cams0), dev(p.lms0), dev(p.obs), dev(p.cam_idx), dev(p.lm_idx),
                           options=poba.ba_default_options(eps=0.0, max_inner=5), stream=s)
        poba.ba_linearize(h)
        poba.ba_solve_schur_power(h, 1e-3)
        out_p = torch.empty((16, 9), dtype=torch.float64, device="cuda")
        out_l = torch.empty((600, 3), dtype=torch.float64, device="cuda")
        poba.ba_get_step(h, out_p, out_l)
    torch.cuda.synchronize()
    o = OracleRef(p).solve(1e-3, 0.0, 5)
    assert rel(out_p.cpu().numpy(), o["x"]) < 1e-10
    assert rel(out_l.cpu().numpy(), o["xl"]) < 1e-10
    check_step_blocks(out_p.cpu().numpy(), out_l.cpu().numpy(), o["x"], o["xl"], 0)


def test_not_spd_is_reported(poba):
    # A camera that nothing observes has U = 0; with lambda = 1e-320 the damping
    # lambda * clamp(0) = lambda * 1e-6 underflows to 0, so its block is not positive definite.
    p = bal_synth.make_problem(4, 50, seed=113)
    p.cams0 = np.vstack([p.cams0, p.cams0[:1]])  # camera 4: no observations -> U = 0
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx,
                       options=poba.ba_default_options(max_inner=2))
    poba.ba_linearize(h)
    with pytest.raises(poba.PobaError) as e:
        poba.ba_solve_schur_power(h, 1e-320)
    assert e.value.status_name == "BA_ERR_NOT_SPD"
    # the handle stays usable
    info = poba.ba_solve_schur_power(h, 1e-3)
    assert info["inner_iters"] >= 0


def test_not_spd_lm_iteration_is_rejected_like_the_oracle(poba):
    """In the LM loop a damped block that fails Cholesky is not an error: the iteration has no
    step, is rejected (state unchanged, lambda raised, here to the 1e-10 clamp) and reports
    not_spd; the following iterations match the oracle's LM loop, which does the same."""
    from oracle import lm as olm
    p = bal_synth.make_problem(4, 60, track=("uniform", 2, 4), seed=113)
    p.cams0 = np.vstack([p.cams0, p.cams0[:1]])  # camera 4: no observations -> U = 0
    _, _, hist = olm.lm_solve(p, olm.Options(lambda0=1e-320, max_lm=6))
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx,
                       options=poba.ba_default_options(lambda0=1e-320, max_lm=6))
    steps = poba.ba_lm_solve(h, max_lm=6)
    assert len(steps) == len(hist)
    s0, o0 = steps[0], hist[0]
    assert s0["not_spd"] and o0["not_spd"] and not s0["accepted"]
    assert np.isnan(s0["cost_after"])
    assert abs(s0["cost_before"] - o0["cost_before"]) <= 1e-12 * o0["cost_before"]
    for s, o in zip(steps[1:], hist[1:]):
        assert not s["not_spd"] and s["accepted"] == o["accepted"] and s["inner"] == o["inner"]
        assert abs(s["lam"] - o["lam"]) <= 1e-12 * o["lam"]
        assert abs(s["cost_after"] - o["cost_after"]) <= 1e-6 * o["cost_after"]
    c, _ = poba.ba_get_params(h)
    assert np.array_equal(c[4], p.cams0[4])


def test_solve_before_linearize(poba):
    p = bal_synth.make_problem(4, 50, seed=115)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    with pytest.raises(poba.PobaError) as e:
        poba.ba_solve_schur_power(h, 1e-3)
    assert e.value.status_name == "BA_ERR_NOT_LINEARIZED"


def test_nonfinite_state_is_reported(poba):
    p = bal_synth.make_problem(4, 50, seed=117)
    cams = p.cams0.copy()
    cams[0, 6] = 1e308  # finite focal length, but |r|^2 overflows to inf
    h = poba.ba_create(cams, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    assert not np.isfinite(poba.ba_cost(h))
    with pytest.raises(poba.PobaError) as e:
        poba.ba_lm_step(h)
    assert e.value.status_name in ("BA_ERR_NONFINITE", "BA_ERR_NOT_SPD")
    # the handle stays usable once the state is repaired
    poba.ba_set_params(h, p.cams0, p.lms0)
    assert np.isfinite(poba.ba_cost(h))


@pytest.mark.parametrize("precision,mode", [(0, 3), (1, 3), (1, 4), (0, 5), (1, 5)])
def test_grid_barrier_timeout_is_reported_and_recoverable(poba, precision, mode):
    """A grid-barrier wait of the persistent series kernel that runs out (limit of one clock
    cycle) makes the solve return BA_ERR_TIMEOUT; the context stays usable and the next solve
    with the normal limit gives the usual result."""
    p = bal_synth.make_problem(40, 2000, track=("uniform", 3, 4), visibility="clustered", seed=119)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=precision,
                       options=poba.ba_default_options(eps=0.0, max_inner=6, series_exec=mode))
    poba.ba_linearize(h)
    ref = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=precision,
                         options=poba.ba_default_options(eps=0.0, max_inner=6, series_exec=1))
    poba.ba_linearize(ref)
    poba.ba_solve_schur_power(ref, 1e-3)
    want = poba.ba_get_step(ref)
    poba.ba_set_barrier_timeout(h, 1)
    with pytest.raises(poba.PobaError) as e:
        poba.ba_solve_schur_power(h, 1e-3)
    assert e.value.status_name == "BA_ERR_TIMEOUT"
    poba.ba_set_barrier_timeout(h, 0)  # back to the default limit
    info = poba.ba_solve_schur_power(h, 1e-3)
    assert info["inner_iters"] == 6
    got = poba.ba_get_step(h)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
