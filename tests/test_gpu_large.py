"""Parity at the large single-problem size (10,000 cameras / 1,000,000 landmarks / about 5.0M
observations, power-law tracks on [2, 50]) in the launch configuration bench.py times (the
autotuned series form).  The oracle cannot run the whole series at this size in seconds, so it
computes sampled outputs one by one: for a camera c, everything that x(0)_c = -U_c^-1 b~_c and
the first term t_1,c = (U^-1 W V^-1 W^T x(0))_c depend on lies in the observations of the
landmarks seen by the cameras that share a landmark with c (Sec. 4.2 and 4.3).  The oracle
builds the normal equation of that subset, which is exact at c, at its neighbours' x(0) and at
every landmark block involved, and evaluates both quantities there."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import rel
from oracle import camera_model as cm
from oracle import normal_eq as neq
from oracle import power_series as ps

pytestmark = pytest.mark.gpu

WORKLOAD = "powerlaw_10000c_1000000l"


@pytest.fixture(scope="module")
def poba():
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    return bal_synth.preset(WORKLOAD)


def local_first_terms(p, cams, lam):
    """Oracle x(0) and t_1 at the cameras `cams` from the sub-problem that determines them."""
    lms_c = np.unique(p.lm_idx[np.isin(p.cam_idx, cams)])
    nbr = np.unique(p.cam_idx[np.isin(p.lm_idx, lms_c)])
    lms_n = np.unique(p.lm_idx[np.isin(p.cam_idx, nbr)])
    sel = np.flatnonzero(np.isin(p.lm_idx, lms_n))
    cu, ci = np.unique(p.cam_idx[sel], return_inverse=True)
    lu, li = np.unique(p.lm_idx[sel], return_inverse=True)
    w = None if p.weights is None else p.weights[sel]
    r, Jp, Jl = cm.linearize(p.cams0[cu], p.lms0[lu], p.obs[sel], ci, li, w)
    ne = neq.NormalEquation(r, Jp, Jl, ci, li, len(cu), len(lu))
    Ul, Vl = ne.damped(lam)
    Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
    x0 = -neq.apply_blocks(Ui, neq.schur_rhs(ne, Vi))
    t1 = ps.apply_P(ne, Ui, Vi, x0)
    k = np.searchsorted(cu, cams)
    return x0.reshape(-1, 9)[k], t1.reshape(-1, 9)[k]


@pytest.fixture(scope="module")
def sampled(problem):
    rng = np.random.default_rng(11)
    cams = np.sort(rng.choice(problem.n_cams, 3, replace=False))
    lam = 1e-4
    x0, t1 = local_first_terms(problem, cams, lam)
    return cams, lam, x0, t1


def gpu_first_terms(poba, p, precision, lam):
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=precision)
    poba.ba_autotune(h, trials=1)
    poba.ba_set_options(h, poba.ba_default_options(eps=0.0, max_inner=0))
    poba.ba_linearize(h, want_cost=False)
    info0 = poba.ba_solve_schur_power(h, lam)
    x0 = poba.ba_get_step(h)[0].reshape(-1, 9).copy()
    poba.ba_set_options(h, poba.ba_default_options(eps=0.0, max_inner=1))
    info1 = poba.ba_solve_schur_power(h, lam)
    x1 = poba.ba_get_step(h)[0].reshape(-1, 9)
    assert info0["inner_iters"] == 0 and info1["inner_iters"] == 1
    return h, x0, x1 - x0


@pytest.mark.parametrize("precision,tol", [(1, 1e-4), (0, 1e-10)])
def test_first_terms_at_sampled_cameras(poba, problem, sampled, precision, tol):
    cams, lam, x0_o, t1_o = sampled
    h, x0, t1 = gpu_first_terms(poba, problem, precision, lam)
    assert np.all(np.isfinite(x0)) and np.all(np.isfinite(t1))
    assert rel(x0[cams], x0_o) < tol, rel(x0[cams], x0_o)
    assert rel(t1[cams], t1_o) < tol, rel(t1[cams], t1_o)
    poba.ba_destroy(h)


def test_lm_decreases_cost(poba, problem):
    """FP32 bulk, three LM iterations from x0 in the tuned form: each accepted step lowers the
    cost, the reported costs agree with ba_cost (to float rounding: the first one may come from
    the FP32 linearisation), and the state stays finite (properties that hold at any size)."""
    p = problem
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=1)
    poba.ba_autotune(h, trials=1)
    poba.ba_set_params(h, p.cams0, p.lms0)
    poba.ba_set_lm_state(h, 1e-4, 2.0, 0)
    f0 = poba.ba_cost(h)
    f = f0
    accepted = 0
    for _ in range(3):
        s = poba.ba_lm_step(h)
        assert s["cost_before"] == pytest.approx(f, rel=1e-6)
        if s["accepted"]:
            assert s["cost_after"] < s["cost_before"]
            f = s["cost_after"]
            accepted += 1
    assert accepted >= 1 and f < f0
    assert poba.ba_cost(h) == pytest.approx(f, rel=1e-6)
    cams, lms = poba.ba_get_params(h)
    assert np.all(np.isfinite(cams)) and np.all(np.isfinite(lms))
    poba.ba_destroy(h)
