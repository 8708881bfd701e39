"""Parity at the benchmark's full size (clustered 1,200 cameras / 160,000 landmarks / 559,912
observations) in the launch configuration bench.py times (persistent series kernel, Sec. 5.1
settings).  Linearisation and blocks are checked on sampled cameras, landmarks and observations
that the oracle computes one by one; the series step is checked against the full oracle series
(about ten seconds of CPU time); two LM iterations are checked against the oracle's LM."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import OracleRef, check_step_blocks, rel
from oracle import camera_model as cm
from oracle import lm as olm

pytestmark = pytest.mark.gpu

WORKLOAD = "clustered_1200c_160000l"


@pytest.fixture(scope="module")
def poba():
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    return bal_synth.preset(WORKLOAD)


@pytest.fixture(scope="module")
def oracle_ref(problem):
    return OracleRef(problem)


def test_sampled_linearization_and_blocks(poba, problem):
    p = problem
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    poba.ba_linearize(h)
    r, Jp, Jl = poba.ba_get_linearization(h)
    U, V, bp, bl = poba.ba_get_blocks(h)
    rng = np.random.default_rng(0)
    obs_s = rng.choice(p.n_obs, 3000, replace=False)
    ro, Jpo, Jlo = cm.linearize(p.cams0, p.lms0, p.obs[obs_s], p.cam_idx[obs_s], p.lm_idx[obs_s])
    assert np.abs(r[obs_s] - ro).max() <= 1e-12 * max(1.0, np.abs(ro).max())
    assert np.abs(Jp[obs_s] - Jpo).max() <= 1e-12 * np.abs(Jpo).max()
    assert np.abs(Jl[obs_s] - Jlo).max() <= 1e-12 * np.abs(Jlo).max()
    for c in rng.choice(p.n_cams, 8, replace=False):
        sel = np.nonzero(p.cam_idx == c)[0]
        rc, Jpc, _ = cm.linearize(p.cams0, p.lms0, p.obs[sel], p.cam_idx[sel], p.lm_idx[sel])
        Uc = np.einsum("oij,oik->jk", Jpc, Jpc)
        bc = np.einsum("oij,oi->j", Jpc, rc)
        assert np.abs(U[c] - Uc).max() <= 1e-12 * np.abs(Uc).max()
        assert np.abs(bp[9 * c:9 * c + 9] - bc).max() <= 1e-10 * max(np.abs(bc).max(), 1e-300)
    for l in rng.choice(p.n_lms, 64, replace=False):
        sel = np.nonzero(p.lm_idx == l)[0]
        rl, _, Jll = cm.linearize(p.cams0, p.lms0, p.obs[sel], p.cam_idx[sel], p.lm_idx[sel])
        Vl = np.einsum("oij,oik->jk", Jll, Jll)
        assert np.abs(V[l] - Vl).max() <= 1e-12 * np.abs(Vl).max()
        bll = np.einsum("oij,oi->j", Jll, rl)
        assert np.abs(bl[3 * l:3 * l + 3] - bll).max() <= 1e-10 * max(np.abs(bll).max(), 1e-12)


@pytest.mark.parametrize("eps,m", [(0.0, 20), (0.01, 20)])
def test_full_series_fp64_and_fp32(poba, problem, oracle_ref, eps, m):
    p = problem
    lam = 1e-4
    o = oracle_ref.solve(lam, eps, m)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=prec,
                           options=poba.ba_default_options(eps=eps, max_inner=m))
        poba.ba_linearize(h)
        info = poba.ba_solve_schur_power(h, lam)
        dxp, dxl = poba.ba_get_step(h)
        if prec == 0:
            assert info["inner_iters"] == o["m"]
        assert rel(dxp, o["x"]) < tol, (prec, rel(dxp, o["x"]))
        assert rel(dxl, o["xl"]) < tol, (prec, rel(dxl, o["xl"]))
        check_step_blocks(dxp, dxl, o["x"], o["xl"], prec)


def test_fp32_persistent_forms_agree_bitwise(poba, problem):
    """FP32-bulk at full size: the persistent kernel (3), its staged-chunk form (4), the
    dataflow form (5), the replayed graph of per-term launches (1) and the handle's choice (2) give the same step bit
    for bit, with the stop rule on."""
    p = problem
    out = []
    for mode in (2, 3, 4, 5, 1):
        h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=1,
                           options=poba.ba_default_options(series_exec=mode))
        poba.ba_linearize(h)
        info = poba.ba_solve_schur_power(h, 1e-2)
        out.append((info["inner_iters"], poba.ba_get_step(h)))
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert np.array_equal(o[1][0], out[0][1][0]) and np.array_equal(o[1][1], out[0][1][1])


def test_two_lm_iterations(poba, problem):
    p = problem
    _, _, hist = olm.lm_solve(p, olm.Options(max_lm=2, func_tol=0.0))
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx,
                       options=poba.ba_default_options(func_tol=0.0))
    for o in hist:
        s = poba.ba_lm_step(h)
        assert s["accepted"] == o["accepted"]
        assert s["inner"] == o["inner"]
        assert abs(s["cost_after"] - o["cost_after"]) <= 1e-6 * o["cost_after"]
