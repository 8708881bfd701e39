"""Pins for the oracle's normal equation, Schur complement and back-substitution (Sec. 4.1,
4.2): brute-force dense J^T J, a full dense H solve, explicit inverses and closed forms."""
import numpy as np
import pytest

import bal_synth
from oracle import camera_model as cm
from oracle import normal_eq as neq
from oracle import direct


def _tiny(seed=11, nc=4, nl=25, weighted=False):
    p = bal_synth.make_problem(nc, nl, track=("uniform", 2, 4), seed=seed, weighted=weighted)
    r, Jp, Jl = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    return p, r, Jp, Jl


def _dense_J(p, Jp, Jl):
    """Dense J = [J_p J_l] written out observation by observation (pure Python loops)."""
    n = p.n_obs
    J = np.zeros((2 * n, 9 * p.n_cams + 3 * p.n_lms))
    for o in range(n):
        c, l = p.cam_idx[o], p.lm_idx[o]
        for i in range(2):
            for j in range(9):
                J[2 * o + i, 9 * c + j] = Jp[o, i, j]
            for j in range(3):
                J[2 * o + i, 9 * p.n_cams + 3 * l + j] = Jl[o, i, j]
    return J


def test_blocks_equal_dense_normal_matrix():
    p, r, Jp, Jl = _tiny(weighted=True)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    J = _dense_J(p, Jp, Jl)
    H = J.T @ J
    b = J.T @ r.ravel()
    npp = 9 * p.n_cams
    for c in range(p.n_cams):
        np.testing.assert_allclose(ne.U[c], H[9 * c:9 * c + 9, 9 * c:9 * c + 9], rtol=1e-13, atol=1e-9)
    for l in range(p.n_lms):
        s = npp + 3 * l
        np.testing.assert_allclose(ne.V[l], H[s:s + 3, s:s + 3], rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(ne.W.toarray(), H[:npp, npp:], rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(ne.b_p, b[:npp], rtol=1e-13, atol=1e-9)
    np.testing.assert_allclose(ne.b_l, b[npp:], rtol=1e-13, atol=1e-9)
    # U is block diagonal: no coupling between different cameras
    off = H[:npp, :npp].copy()
    for c in range(p.n_cams):
        off[9 * c:9 * c + 9, 9 * c:9 * c + 9] = 0
    assert np.abs(off).max() == 0.0


def test_damping_modes():
    A = np.array([[[4.0, 1.0], [1.0, 0.0]]])
    D0 = neq.damp(A, 0.5, 0)
    np.testing.assert_allclose(D0[0], [[4.0 + 2.0, 1.0], [1.0, 0.5 * neq.DAMP_MIN]], rtol=1e-15, atol=0)
    D1 = neq.damp(A, 0.5, 1)
    np.testing.assert_allclose(D1[0], [[4.5, 1.0], [1.0, 0.5]], rtol=0, atol=0)


def test_block_cholesky_inverse():
    p, r, Jp, Jl = _tiny()
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    Ul, Vl = ne.damped(1e-4)
    Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
    for c in range(p.n_cams):
        np.testing.assert_allclose(Ui[c] @ Ul[c], np.eye(9), rtol=0, atol=1e-9)
    for l in range(p.n_lms):
        np.testing.assert_allclose(Vi[l] @ Vl[l], np.eye(3), rtol=0, atol=1e-10)
    # an undamped zero block is not positive definite
    with pytest.raises(np.linalg.LinAlgError):
        neq.chol_inverse(np.zeros((1, 3, 3)))


@pytest.mark.parametrize("lam,mode", [(1e-4, 0), (1.0, 0), (1e-2, 1)])
def test_schur_route_equals_full_dense_solve(lam, mode):
    """dx from S dx_p = -b~ plus back-substitution equals H^-1 (-b) for the dense H (pins the
    derived sign of the back-substitution)."""
    p, r, Jp, Jl = _tiny(seed=13)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    J = _dense_J(p, Jp, Jl)
    H = J.T @ J
    d = np.diag(H).copy()
    H[np.diag_indices_from(H)] += lam * (np.clip(d, neq.DAMP_MIN, neq.DAMP_MAX) if mode == 0 else 1.0)
    dx_ref = np.linalg.solve(H, -(J.T @ r.ravel()))
    Ul, Vl = ne.damped(lam, mode)
    Vi = neq.chol_inverse(Vl)
    bt = neq.schur_rhs(ne, Vi)
    S = neq.explicit_schur(ne, Ul, Vi, dense=True)
    dx_p = direct.solve_dense(S, bt)
    dx_l = neq.back_substitute(ne, Vi, dx_p)
    dx = np.concatenate([dx_p, dx_l])
    assert np.linalg.norm(dx - dx_ref) / np.linalg.norm(dx_ref) < 1e-9
    # the explicit S is the dense Schur complement of H
    npp = 9 * p.n_cams
    S_ref = H[:npp, :npp] - H[:npp, npp:] @ np.linalg.solve(H[npp:, npp:], H[npp:, :npp])
    np.testing.assert_allclose(S, S_ref, rtol=1e-9, atol=1e-6 * np.abs(S_ref).max())
    # S is symmetric positive definite (Sec. 4.1, lambda > 0)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-9 * np.abs(S).max())
    assert np.linalg.eigvalsh(S).min() > 0


def test_pcg_matches_dense_cholesky():
    p = bal_synth.make_problem(30, 600, track=("uniform", 3, 5), visibility="clustered", seed=21)
    r, Jp, Jl = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    Ul, Vl = ne.damped(1e-3)
    Vi = neq.chol_inverse(Vl)
    bt = neq.schur_rhs(ne, Vi)
    x_dense = direct.solve_dense(neq.explicit_schur(ne, Ul, Vi, True), bt)
    S = neq.explicit_schur(ne, Ul, Vi, dense=False)
    Minv = neq.chol_inverse(neq.block_diagonal(S, p.n_cams, 9))
    y, it, rel = direct.pcg(S, -bt, Minv, rtol=1e-13)
    assert rel < 1e-12
    assert np.linalg.norm(y - x_dense) / np.linalg.norm(x_dense) < 1e-8


def test_model_decrease_closed_form():
    p, r, Jp, Jl = _tiny(seed=17)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    rng = np.random.default_rng(0)
    dxp = rng.normal(size=9 * p.n_cams) * 1e-3
    dxl = rng.normal(size=3 * p.n_lms) * 1e-3
    J = _dense_J(p, Jp, Jl)
    dx = np.concatenate([dxp, dxl])
    b = J.T @ r.ravel()
    ref = -(b @ dx) - 0.5 * dx @ (J.T @ J) @ dx
    np.testing.assert_allclose(neq.model_decrease(ne, dxp, dxl), ref, rtol=1e-8)


def test_solve_reduced_takes_pcg_above_the_dense_limit():
    """Above 9 n_c = DENSE_LIMIT the exact reduced solve switches from dense Cholesky to PCG on
    the explicit block-sparse S; its dx_p solves S dx_p = -b~ like the dense route."""
    p = bal_synth.make_problem(240, 3000, track=("uniform", 3, 5), visibility="clustered", seed=23)
    assert 9 * p.n_cams > direct.DENSE_LIMIT
    r, Jp, Jl = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    Ul, Vl = ne.damped(1e-3)
    Vi = neq.chol_inverse(Vl)
    bt = neq.schur_rhs(ne, Vi)
    dx = direct.solve_reduced(ne, Ul, Vi, bt)
    S = neq.explicit_schur(ne, Ul, Vi, dense=True)
    x_dense = direct.solve_dense(S, bt)
    assert np.linalg.norm(S @ dx + bt) / np.linalg.norm(bt) < 1e-11
    assert np.linalg.norm(dx - x_dense) / np.linalg.norm(x_dense) < 1e-8
