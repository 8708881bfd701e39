"""GPU LM loop against the oracle's LM loop (Sec. 5.1 settings): same accept / reject
decisions, final cost within 1e-6 relative; checkpoint / resume reproduces the trajectory."""
import numpy as np
import pytest

import bal_synth
from oracle import lm as olm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def poba():
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    return m


def run_gpu(poba, p, n_iter, precision=0, **opt):
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights,
                       precision=precision, options=poba.ba_default_options(**opt))
    steps = []
    for _ in range(n_iter):
        s = poba.ba_lm_step(h)
        steps.append(s)
        if s["converged"]:
            break
    return h, steps


def test_lm_20_iterations_small_problem_fp64(poba):
    """16 cameras, 1,000 landmarks, 20 LM iterations, series truncated at eps = 1e-10."""
    p = bal_synth.preset("uniform_16c_1000l")
    opts = olm.Options(max_lm=20, eps=1e-10, func_tol=0.0)
    cams, lms, hist = olm.lm_solve(p, opts)
    h, steps = run_gpu(poba, p, 20, eps=1e-10, func_tol=0.0)
    assert len(steps) == len(hist)
    for s, o in zip(steps, hist):
        assert s["accepted"] == o["accepted"]
        assert s["inner"] == o["inner"]
        assert abs(s["cost_after"] - o["cost_after"]) <= 1e-6 * o["cost_after"]
        assert abs(s["lam"] - o["lam"]) <= 1e-6 * o["lam"]
    f_gpu = poba.ba_cost(h)
    f_orc = min(e["cost_after"] for e in hist if e["accepted"])
    assert abs(f_gpu - f_orc) <= 1e-6 * f_orc
    c, l = poba.ba_get_params(h)
    assert np.abs(c - cams).max() < 1e-6 * np.abs(cams).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_lm_default_settings_reach_oracle_cost(poba, precision):
    p = bal_synth.make_problem(40, 3000, track=("uniform", 3, 4), visibility="clustered", seed=91)
    cams, lms, hist = olm.lm_solve(p, olm.Options(max_lm=25))
    f0 = hist[0]["cost_before"]
    f_orc = min(e["cost_after"] for e in hist if e["accepted"])
    h, steps = run_gpu(poba, p, 25, precision=precision)
    f_gpu = poba.ba_cost(h)
    if precision == 0:
        assert abs(f_gpu - f_orc) <= 1e-6 * f_orc
    else:
        # FP32-bulk: within the tau = 1% band of the FP64 oracle's reduction
        assert f_gpu <= f_orc + 0.01 * (f0 - f_orc)
    for s in steps:
        if s["accepted"]:
            assert s["cost_after"] < s["cost_before"]


def test_weighted_lm(poba):
    p = bal_synth.make_problem(30, 1500, track=("uniform", 2, 6), weighted=True, seed=93)
    _, _, hist = olm.lm_solve(p, olm.Options(max_lm=10, func_tol=0.0))
    h, steps = run_gpu(poba, p, 10, func_tol=0.0)
    for s, o in zip(steps, hist):
        assert s["accepted"] == o["accepted"]
        assert abs(s["cost_after"] - o["cost_after"]) <= 1e-6 * o["cost_after"]


def test_checkpoint_resume_is_bitwise(poba):
    p = bal_synth.make_problem(20, 800, seed=95)
    h, steps = run_gpu(poba, p, 8, func_tol=0.0)
    ref = steps[4:]
    h2, first = run_gpu(poba, p, 4, func_tol=0.0)
    cams, lms = poba.ba_get_params(h2)
    st = poba.ba_get_lm_state(h2)
    h3 = poba.ba_create(cams, lms, p.obs, p.cam_idx, p.lm_idx, options=poba.ba_default_options(func_tol=0.0))
    poba.ba_set_lm_state(h3, st["lam"], st["nu"], st["iteration"])
    for r in ref:
        s = poba.ba_lm_step(h3)
        assert s["accepted"] == r["accepted"]
        assert s["cost_after"] == r["cost_after"]
        assert s["lam"] == r["lam"]
        assert s["it"] == r["it"]
    a, b = poba.ba_get_params(h), poba.ba_get_params(h3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_lm_solve_entry_point(poba):
    p = bal_synth.make_problem(10, 300, seed=97)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx,
                       options=poba.ba_default_options(max_lm=30))
    trace = poba.ba_lm_solve(h, 30)
    assert 1 <= len(trace) <= 30
    assert trace[-1]["converged"] or len(trace) == 30
    _, _, hist = olm.lm_solve(p, olm.Options(max_lm=30))
    assert len(trace) == len(hist)


@pytest.mark.parametrize("precision", [0, 1])
def test_state_round_trip_keeps_the_linearisation(poba, precision):
    """ba_set_params with the state ba_get_params returned (bit for bit) changes nothing: the
    linearisation stays in place (no relinearisation after a rejected step), and an LM run that
    passes its state through the host every step gives the device loop's steps and final state
    bit for bit.  A state that differs in one bit marks the linearisation stale."""
    p = bal_synth.make_problem(60, 3000, track=("uniform", 2, 6), visibility="clustered",
                               seed=131)
    opt = poba.ba_default_options(func_tol=0.0)
    h1 = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, options=opt,
                        precision=precision)
    h2 = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, options=opt,
                        precision=precision)
    s1, s2 = [], []
    for _ in range(25):
        s1.append(poba.ba_lm_step(h1))
        c, l = poba.ba_get_params(h2)
        poba.ba_set_params(h2, c, l)
        s2.append(poba.ba_lm_step(h2))
    for a, b in zip(s1, s2):
        assert a["accepted"] == b["accepted"] and a["cost_after"] == b["cost_after"]
    c1, l1 = poba.ba_get_params(h1)
    c2, l2 = poba.ba_get_params(h2)
    assert np.array_equal(c1, c2) and np.array_equal(l1, l2)
    # the linearisation survives a round trip of the current state
    poba.ba_linearize(h2)
    c, l = poba.ba_get_params(h2)
    poba.ba_set_params(h2, c, l)
    poba.ba_get_linearization(h2)
    # and goes stale when one value changes in its last bit
    l = l.copy()
    l[5, 1] = np.nextafter(l[5, 1], np.inf)
    poba.ba_set_params(h2, c, l)
    with pytest.raises(poba.PobaError) as e:
        poba.ba_get_linearization(h2)
    assert e.value.status_name == "BA_ERR_NOT_LINEARIZED"
