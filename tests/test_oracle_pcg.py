"""Pins for the oracle's preconditioned conjugate gradients (oracle/pcg.py): convergence to the
exact reduced solve with both preconditioners, the special cases where a preconditioner is the
exact inverse (single-observation tracks make S block diagonal, so Schur-Jacobi PCG finishes in
one iteration; a long power series approaches S^-1), and the order-0 power series being the
U^-1 block preconditioner."""
import numpy as np
import pytest

import bal_synth
from oracle import camera_model as cm
from oracle import normal_eq as neq
from oracle import pcg as opcg
from oracle.direct import solve_dense


def normal_eq(p):
    r, Jp, Jl = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    return neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)


def exact(ne, lam):
    Ul, Vl = ne.damped(lam)
    Vi = neq.chol_inverse(Vl)
    return solve_dense(neq.explicit_schur(ne, Ul, Vi), neq.schur_rhs(ne, Vi))


@pytest.mark.parametrize("precond,m", [("jacobi", 0), ("power", 1), ("power", 3)])
def test_pcg_converges_to_the_exact_reduced_solve(precond, m):
    p = bal_synth.make_problem(12, 300, track=("uniform", 2, 6), weighted=True, seed=401)
    ne = normal_eq(p)
    lam = 1e-3
    dx, dxl, it, relres = opcg.pcg_solve(ne, lam, precond, m, rtol=1e-12, max_iter=2000)
    assert relres <= 1e-12 and it < 2000
    x = exact(ne, lam)
    assert np.linalg.norm(dx - x) <= 1e-8 * np.linalg.norm(x)
    Ul, Vl = ne.damped(lam)
    assert np.allclose(dxl, neq.back_substitute(ne, neq.chol_inverse(Vl), dx), rtol=0, atol=1e-12 * np.abs(dxl).max())


def test_schur_jacobi_is_exact_for_single_observation_tracks():
    """Each landmark seen once: W V^-1 W^T only touches its camera's block, S is block diagonal
    and Schur-Jacobi PCG solves the system in one iteration."""
    p = bal_synth.make_problem(8, 200, track=("uniform", 1, 1), seed=403)
    assert np.all(np.bincount(p.lm_idx, minlength=p.n_lms) == 1)
    ne = normal_eq(p)
    dx, _, it, relres = opcg.pcg_solve(ne, 1e-2, "jacobi", rtol=1e-12)
    assert it == 1 and relres <= 1e-12
    x = exact(ne, 1e-2)
    assert np.linalg.norm(dx - x) <= 1e-10 * np.linalg.norm(x)


def test_long_power_series_preconditioner_approaches_the_inverse():
    p = bal_synth.make_problem(10, 200, track=("uniform", 2, 5), seed=405)
    ne = normal_eq(p)
    lam = 1.0  # spectral radius of P well below 1: the series converges quickly
    its = [opcg.pcg_solve(ne, lam, "power", m, rtol=1e-10)[2] for m in (0, 2, 8, 60)]
    assert its[-1] == 1
    assert its[0] >= its[1] >= its[2] >= its[3]


def test_order_zero_power_series_is_the_U_block_preconditioner():
    p = bal_synth.make_problem(10, 200, track=("uniform", 2, 5), seed=407)
    ne = normal_eq(p)
    lam = 1e-2
    Ul, Vl = ne.damped(lam)
    Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
    r = np.random.default_rng(0).normal(size=9 * p.n_cams)
    z = opcg.power_series_preconditioner(ne, Ui, Vi, 0)(r)
    assert np.array_equal(z, neq.apply_blocks(Ui, r))
    # and one term adds P U^-1 r = U^-1 W V^-1 W^T U^-1 r
    z1 = opcg.power_series_preconditioner(ne, Ui, Vi, 1)(r)
    t = neq.apply_blocks(Ui, r)
    assert np.allclose(z1 - z, neq.apply_blocks(Ui, ne.W @ neq.apply_blocks(Vi, ne.W.T @ t)),
                       rtol=1e-12, atol=1e-14 * np.abs(z1).max())
