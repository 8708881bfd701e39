"""GPU preconditioned conjugate gradients on the reduced camera system (Schur-Jacobi and the
power-series preconditioner) against the oracle (oracle/pcg.py) and the exact reduced solve."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import OracleRef, rel
from oracle import normal_eq as neq
from oracle import pcg as opcg
from oracle.direct import solve_dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def poba():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    m.library()
    return m


@pytest.fixture(scope="module")
def case():
    p = bal_synth.make_problem(30, 800, track=("uniform", 2, 6), weighted=True,
                               visibility="clustered", seed=501)
    return p, OracleRef(p)


def exact_step(ref, lam):
    Ul, Vl = ref.ne.damped(lam)
    Vi = neq.chol_inverse(Vl)
    x = solve_dense(neq.explicit_schur(ref.ne, Ul, Vi), neq.schur_rhs(ref.ne, Vi))
    return x, neq.back_substitute(ref.ne, Vi, x)


def handle(poba, p, precision=0, **opt):
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights, precision=precision,
                       options=poba.ba_default_options(**opt))
    poba.ba_linearize(h)
    return h


@pytest.mark.parametrize("precond,m", [("jacobi", 0), ("power", 1), ("power", 3)])
def test_pcg_matches_oracle_and_exact_solve(poba, case, precond, m):
    p, ref = case
    lam = 1e-3
    h = handle(poba, p)
    info = poba.ba_solve_schur_pcg(h, lam, precond, m, rtol=1e-12, max_iter=3000)
    assert info["converged"] and info["rel_residual"] <= 1e-12
    dxp, dxl = poba.ba_get_step(h)
    _, _, it_o, _ = opcg.pcg_solve(ref.ne, lam, precond, m, rtol=1e-12, max_iter=3000)
    assert abs(info["iterations"] - it_o) <= 2, (info["iterations"], it_o)
    x, xl = exact_step(ref, lam)
    assert rel(dxp, x) < 1e-8 and rel(dxl, xl) < 1e-8


def test_pcg_first_iterates_match_oracle(poba, case):
    """A fixed number of iterations (no convergence test): the same iterate as the oracle."""
    p, ref = case
    for precond, m in (("jacobi", 0), ("power", 2)):
        h = handle(poba, p)
        info = poba.ba_solve_schur_pcg(h, 1e-2, precond, m, rtol=0.0, max_iter=6)
        assert info["iterations"] == 6 and not info["converged"]
        dxp, _ = poba.ba_get_step(h)
        xo, _, it, _ = opcg.pcg_solve(ref.ne, 1e-2, precond, m, rtol=0.0, max_iter=6)
        assert it == 6
        assert rel(dxp, xo) < 1e-10


def test_schur_jacobi_one_iteration_for_single_observation_tracks(poba):
    p = bal_synth.make_problem(8, 200, track=("uniform", 1, 1), seed=503)
    ref = OracleRef(p)
    h = handle(poba, p)
    info = poba.ba_solve_schur_pcg(h, 1e-2, "jacobi", rtol=1e-12)
    assert info["iterations"] == 1 and info["converged"]
    x, xl = exact_step(ref, 1e-2)
    dxp, dxl = poba.ba_get_step(h)
    assert rel(dxp, x) < 1e-10 and rel(dxl, xl) < 1e-10


def schur_cancellation(ne, lam):
    """||(|U_lam| + |W| |V_lam^-1| |W|^T) t|| / ||S t|| at t = 1: how many digits the float
    products lose when S t = U_lam t - W V_lam^-1 W^T t cancels."""
    Ul, Vl = ne.damped(lam)
    Vi = neq.chol_inverse(Vl)
    t = np.ones(9 * ne.n_cams)
    aW = abs(ne.W)
    mag = neq.apply_blocks(np.abs(Ul), t) + aW @ neq.apply_blocks(np.abs(Vi), aW.T @ t)
    return float(np.linalg.norm(mag) / np.linalg.norm(opcg.schur_apply(ne, Ul, Vi, t)))


def test_pcg_fp32_bulk(poba, case):
    """FP32-bulk: the same iterates as the oracle's FP64 PCG for a fixed number of iterations;
    a converged solve takes about as many iterations as in FP64.  The bound follows from the
    arithmetic: a float S p carries about one float rounding (2^-24) times the cancellation
    ratio of U_lam - W V^-1 W^T (about 8e3 here at lambda = 1e-2) and CG passes it on to the
    iterate, so the test allows twice that.  (The converged FP32 step solves the float system:
    its FP64 residual is bounded by cond(S) times the float rounding of J, not by rtol.)"""
    p, ref = case
    tol = 2.0 * schur_cancellation(ref.ne, 1e-2) * 2.0 ** -24
    assert 1e-4 < tol < 2e-3
    for precond, m in (("jacobi", 0), ("power", 2)):
        h = handle(poba, p, precision=1)
        poba.ba_solve_schur_pcg(h, 1e-2, precond, m, rtol=0.0, max_iter=6)
        dxp, _ = poba.ba_get_step(h)
        xo, _, _, _ = opcg.pcg_solve(ref.ne, 1e-2, precond, m, rtol=0.0, max_iter=6)
        assert rel(dxp, xo) < tol, (precond, rel(dxp, xo), tol)
    h = handle(poba, p, precision=1)
    info = poba.ba_solve_schur_pcg(h, 1e-3, "jacobi", rtol=1e-6, max_iter=1000)
    h64 = handle(poba, p)
    info64 = poba.ba_solve_schur_pcg(h64, 1e-3, "jacobi", rtol=1e-6, max_iter=1000)
    assert info["converged"] and info64["converged"]
    assert abs(info["iterations"] - info64["iterations"]) <= 0.2 * info64["iterations"] + 2


def test_power_preconditioner_is_independent_of_series_form(poba, case):
    p, _ = case
    out = []
    for mode in (0, 1, 3):
        h = handle(poba, p, series_exec=mode)
        info = poba.ba_solve_schur_pcg(h, 1e-2, "power", 2, rtol=1e-9, max_iter=200)
        out.append((info["iterations"], poba.ba_get_step(h)))
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert np.array_equal(o[1][0], out[0][1][0]) and np.array_equal(o[1][1], out[0][1][1])
