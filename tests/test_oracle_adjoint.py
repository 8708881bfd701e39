"""Pins for the oracle's implicit-differentiation adjoint (oracle/adjoint.py).  Each test checks
the adjoint gradients against finite differences of a separate computation -- a damped Gauss-
Newton step formed with the full dense H (no Schur complement), or a re-solved regularised
minimiser -- following the statements of that module's docstring."""
import numpy as np
import pytest

import bal_synth
from oracle import adjoint as oad
from oracle import camera_model as cm
from oracle import normal_eq as neq


def dense_step(p, cams, lms, obs, weights, lam, damping_mode=0):
    """dx = -H_lam^-1 J^T W r with the full dense H_lam = J^T W J + lam D^T D (no Schur)."""
    r, Jp, Jl = cm.linearize(cams, lms, obs, p.cam_idx, p.lm_idx, weights)
    Jps, Jls = neq.assemble_jacobians(Jp, Jl, p.cam_idx, p.lm_idx, cams.shape[0], lms.shape[0])
    J = np.hstack([Jps.toarray(), Jls.toarray()])
    H = J.T @ J
    d = np.diag(H).copy()
    if damping_mode == 0:
        d = np.clip(d, neq.DAMP_MIN, neq.DAMP_MAX)
    else:
        d = np.ones_like(d)
    H[np.diag_indices_from(H)] += lam * d
    return -np.linalg.solve(H, J.T @ r.ravel())


def random_gradient(p, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(p.n_cams, 9)), rng.normal(size=(p.n_lms, 3))


def test_obs_gradient_is_the_derivative_of_a_damped_step():
    """At any linearisation point, g^T dx(obs) is linear in obs and its gradient is w J a."""
    p = bal_synth.make_problem(6, 60, track=("uniform", 2, 5), weighted=True, seed=201)
    lam = 1e-2
    g_c, g_l = random_gradient(p, 1)
    g = np.concatenate([g_c.ravel(), g_l.ravel()])
    d_obs, _, _, _, _ = oad.gradients(p, p.cams0, p.lms0, g_c, g_l, lam)
    rng = np.random.default_rng(2)
    h = 1e-2
    for o in rng.choice(p.n_obs, 12, replace=False):
        for i in range(2):
            ob = p.obs.copy()
            ob[o, i] += h
            fp = g @ dense_step(p, p.cams0, p.lms0, ob, p.weights, lam)
            ob[o, i] -= 2 * h
            fm = g @ dense_step(p, p.cams0, p.lms0, ob, p.weights, lam)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - d_obs[o, i]) <= 1e-7 * max(abs(fd), 1e-3 * np.abs(d_obs).max())


def refined_minimiser(p, iters=40, lam=1e-9):
    """A minimiser of F with ||J^T W r|| at rounding level: damped Gauss-Newton on the dense H."""
    cams, lms = p.cams0.copy(), p.lms0.copy()
    nc = p.n_cams
    for _ in range(iters):
        dx = dense_step(p, cams, lms, p.obs, p.weights, lam)
        cams = cams + dx[: 9 * nc].reshape(nc, 9)
        lms = lms + dx[9 * nc:].reshape(-1, 3)
    return cams, lms


def test_weight_gradient_at_the_optimum():
    """Where J^T W r = 0, the gradient of g^T dx(w) for the damped step is -r^T J a."""
    p = bal_synth.make_problem(6, 60, track=("uniform", 3, 5), weighted=True, seed=203)
    cams, lms = refined_minimiser(p)
    r, Jp, Jl = cm.linearize(cams, lms, p.obs, p.cam_idx, p.lm_idx, p.weights)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    grad = np.concatenate([ne.b_p, ne.b_l])
    assert np.linalg.norm(grad) < 1e-9 * np.linalg.norm(np.abs(Jp).max() * np.abs(r).max() + 1)
    lam = 1e-2
    g_c, g_l = random_gradient(p, 3)
    g = np.concatenate([g_c.ravel(), g_l.ravel()])
    _, d_w, _, _, _ = oad.gradients(p, cams, lms, g_c, g_l, lam)
    rng = np.random.default_rng(4)
    for o in rng.choice(p.n_obs, 12, replace=False):
        h = 1e-4 * p.weights[o]
        w = p.weights.copy()
        w[o] += h
        fp = g @ dense_step(p, cams, lms, p.obs, w, lam)
        w[o] -= 2 * h
        fm = g @ dense_step(p, cams, lms, p.obs, w, lam)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - d_w[o]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(d_w).max())


def regularised_minimiser(p, obs, x0_cams, x0_lms, lam, D2, iters=30):
    """argmin_x F(x; obs) + lam/2 ||D (x - x0)||^2 by Gauss-Newton from x0 (D fixed)."""
    cams, lms = x0_cams.copy(), x0_lms.copy()
    nc = p.n_cams
    x0 = np.concatenate([x0_cams.ravel(), x0_lms.ravel()])
    for _ in range(iters):
        r, Jp, Jl = cm.linearize(cams, lms, obs, p.cam_idx, p.lm_idx, p.weights)
        Jps, Jls = neq.assemble_jacobians(Jp, Jl, p.cam_idx, p.lm_idx, nc, p.n_lms)
        J = np.hstack([Jps.toarray(), Jls.toarray()])
        x = np.concatenate([cams.ravel(), lms.ravel()])
        H = J.T @ J + lam * np.diag(D2)
        rhs = J.T @ r.ravel() + lam * D2 * (x - x0)
        dx = -np.linalg.solve(H, rhs)
        cams = cams + dx[: 9 * nc].reshape(nc, 9)
        lms = lms + dx[9 * nc:].reshape(-1, 3)
    return np.concatenate([cams.ravel(), lms.ravel()])


def test_obs_gradient_of_the_regularised_minimiser_without_noise():
    """With noise-free observations the ground truth has r = 0, Gauss-Newton is the exact
    Hessian there, and the adjoint gradient equals the finite difference of the minimiser of
    F + lam/2 ||D (x - x_gt)||^2 (the prior that fixes the gauge)."""
    p = bal_synth.make_problem(5, 40, track=("uniform", 3, 5), pixel_noise=0.0, seed=205)
    cams, lms = p.cams_gt, p.lms_gt
    assert cm.cost(cams, lms, p.obs, p.cam_idx, p.lm_idx) < 1e-18
    lam = 1e-2
    r, Jp, Jl = cm.linearize(cams, lms, p.obs, p.cam_idx, p.lm_idx, p.weights)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    D2 = np.concatenate([np.clip(ne.U[:, np.arange(9), np.arange(9)], neq.DAMP_MIN, neq.DAMP_MAX).ravel(),
                         np.clip(ne.V[:, np.arange(3), np.arange(3)], neq.DAMP_MIN, neq.DAMP_MAX).ravel()])
    g_c, g_l = random_gradient(p, 5)
    g = np.concatenate([g_c.ravel(), g_l.ravel()])
    d_obs, d_w, _, _, _ = oad.gradients(p, cams, lms, g_c, g_l, lam)
    assert np.abs(d_w).max() < 1e-12 * np.abs(d_obs).max()  # r = 0
    rng = np.random.default_rng(6)
    h = 1e-4
    for o in rng.choice(p.n_obs, 8, replace=False):
        for i in range(2):
            ob = p.obs.copy()
            ob[o, i] += h
            fp = g @ regularised_minimiser(p, ob, cams, lms, lam, D2)
            ob[o, i] -= 2 * h
            fm = g @ regularised_minimiser(p, ob, cams, lms, lam, D2)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - d_obs[o, i]) <= 1e-5 * max(abs(fd), 1e-2 * np.abs(d_obs).max())


@pytest.mark.parametrize("lam", [1e-1, 1.0])
def test_power_series_adjoint_converges_to_the_direct_one(lam):
    """The adjoint solved with the truncated series approaches the exact reduced solve as the
    series lengthens (Prop. 2), and the stop rule's m is reported."""
    p = bal_synth.make_problem(8, 120, track=("uniform", 2, 5), seed=207)
    g_c, g_l = random_gradient(p, 7)
    exact = oad.gradients(p, p.cams0, p.lms0, g_c, g_l, lam)
    prev = None
    for m in (5, 20, 80, 400):
        approx = oad.gradients(p, p.cams0, p.lms0, g_c, g_l, lam, solver="power", eps=0.0, m_max=m)
        assert approx[4] == m
        err = np.linalg.norm(approx[0] - exact[0]) / np.linalg.norm(exact[0])
        if prev is not None:
            assert err < prev or err < 1e-13
        prev = err
    assert prev < 1e-12
