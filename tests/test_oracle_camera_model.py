"""Pins for the oracle's camera model (Sec. 4, BAL convention): hand-computed projections,
finite-difference Jacobians, rotation invariants and the generator's independent projection."""
import json
import os

import numpy as np
import pytest

import bal_synth
from oracle import camera_model as cm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "projection_cases.json")


def _proj(cam, X):
    cam = np.asarray(cam, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    pi = cm.project([np.array([c]) for c in cam], [np.array([x]) for x in X])
    return np.array([pi[0][0], pi[1][0]])


def test_golden_projections():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        np.testing.assert_allclose(_proj(c["cam"], c["X"]), c["pi"], rtol=0, atol=1e-9, err_msg=c["why"])


def test_rotation_preserves_norm_and_inverts():
    rng = np.random.default_rng(0)
    w = rng.normal(0, 1.0, size=(50, 3))
    X = rng.normal(0, 3.0, size=(50, 3))
    RX = cm.rotate([w[:, i] for i in range(3)], [X[:, i] for i in range(3)])
    RX = np.stack(RX, 1)
    np.testing.assert_allclose(np.linalg.norm(RX, axis=1), np.linalg.norm(X, axis=1), rtol=1e-13)
    back = np.stack(cm.rotate([-w[:, i] for i in range(3)], [RX[:, i] for i in range(3)]), 1)
    np.testing.assert_allclose(back, X, rtol=0, atol=1e-12)
    # rotation by theta about z is the planar rotation of (x, y)
    th = 0.7
    r = np.stack(cm.rotate([np.zeros(1), np.zeros(1), np.full(1, th)], [np.ones(1), np.full(1, 2.0), np.full(1, -3.0)]), 1)[0]
    np.testing.assert_allclose(r, [np.cos(th) - 2 * np.sin(th), np.sin(th) + 2 * np.cos(th), -3.0], rtol=0, atol=1e-14)


def test_small_angle_branch_is_continuous():
    X = [np.array([1.0]), np.array([-2.0]), np.array([-7.0])]
    eps = cm.THETA2_SMALL
    for scale in (0.5, 2.0):
        th = np.sqrt(eps * scale)
        w = [np.array([th]), np.array([0.0]), np.array([0.0])]
        RX = np.array([v[0] for v in cm.rotate(w, X)])
        exact = np.array([1.0, -2.0 * np.cos(th) + 7.0 * np.sin(th), -2.0 * np.sin(th) - 7.0 * np.cos(th)])
        np.testing.assert_allclose(RX, exact, rtol=0, atol=1e-14)


def test_jacobians_match_central_differences():
    p = bal_synth.make_problem(5, 40, seed=7)
    cams, lms = p.cams0, p.lms0
    r, Jp, Jl = cm.linearize(cams, lms, p.obs, p.cam_idx, p.lm_idx)
    args = (p.obs, p.cam_idx, p.lm_idx)
    for o in [0, 3, 17, p.n_obs - 1]:
        c, l = p.cam_idx[o], p.lm_idx[o]
        for j in range(12):
            cp, lp = cams.copy(), lms.copy()
            cmn, lmn = cams.copy(), lms.copy()
            val = cams[c, j] if j < 9 else lms[l, j - 9]
            h = 1e-6 * max(1.0, abs(val))
            if j < 9:
                cp[c, j] += h
                cmn[c, j] -= h
            else:
                lp[l, j - 9] += h
                lmn[l, j - 9] -= h
            fd = (cm.residuals(cp, lp, *args)[o] - cm.residuals(cmn, lmn, *args)[o]) / (2 * h)
            an = Jp[o, :, j] if j < 9 else Jl[o, :, j - 9]
            scale = max(1.0, np.abs(an).max())
            assert np.abs(fd - an).max() / scale < 1e-6, (o, j, fd, an)


def test_jacobian_entries_closed_form_at_identity():
    # w = 0, k = 0: pi = -f (X + t)_xy / (X + t)_z.  d pi_x / d t_x = -f / P_z,
    # d pi_x / d t_z = f P_x / P_z^2, d pi_x / d f = -P_x / P_z, and d/dX = d/dt.
    cams = np.array([[0, 0, 0, 0.5, -0.25, 1.0, 400.0, 0, 0]], dtype=np.float64)
    lms = np.array([[1.0, 2.0, -9.0]])
    obs = np.zeros((1, 2))
    r, Jp, Jl = cm.linearize(cams, lms, obs, np.zeros(1, np.int32), np.zeros(1, np.int32))
    P = np.array([1.5, 1.75, -8.0])
    f = 400.0
    np.testing.assert_allclose(Jp[0, 0, 3], -f / P[2], rtol=1e-14)
    np.testing.assert_allclose(Jp[0, 0, 5], f * P[0] / P[2] ** 2, rtol=1e-14)
    np.testing.assert_allclose(Jp[0, 1, 4], -f / P[2], rtol=1e-14)
    np.testing.assert_allclose(Jp[0, 0, 6], -P[0] / P[2], rtol=1e-14)
    np.testing.assert_allclose(Jl[0], Jp[0, :, 3:6], rtol=1e-14)
    # d pi / d k1 = f |p|^2 p at k = 0
    p = -P[:2] / P[2]
    np.testing.assert_allclose(Jp[0, :, 7], f * (p @ p) * p, rtol=1e-13)
    np.testing.assert_allclose(Jp[0, :, 8], f * (p @ p) ** 2 * p, rtol=1e-13)
    # rotation about w at 0: d(RX)/dw = -[X]x, so d pi / d w_z moves x by -X_y
    np.testing.assert_allclose(Jp[0, 0, 2], (-f / P[2]) * (-lms[0, 1]), rtol=1e-12)


def test_generator_noise_is_the_residual_at_ground_truth():
    # The generator synthesises observations with its own (matrix-form) projection; the
    # oracle's residual at the ground truth must give back exactly the injected noise.
    p = bal_synth.make_problem(12, 300, seed=3)
    rg = cm.residuals(p.cams_gt, p.lms_gt, p.obs, p.cam_idx, p.lm_idx)
    np.testing.assert_allclose(rg, -p.noise, rtol=0, atol=1e-9)


def test_weighted_cost():
    p = bal_synth.make_problem(6, 60, seed=5, weighted=True)
    r0 = cm.residuals(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    F = cm.cost(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    np.testing.assert_allclose(F, 0.5 * np.sum(p.weights * np.sum(r0 * r0, 1)), rtol=1e-13)
    rw, Jpw, Jlw = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    r1, Jp1, Jl1 = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    sw = np.sqrt(p.weights)
    np.testing.assert_allclose(rw, r1 * sw[:, None], rtol=1e-14)
    np.testing.assert_allclose(Jpw, Jp1 * sw[:, None, None], rtol=1e-14)


def test_rotation_matches_the_matrix_exponential():
    """R(w) = exp([w]_x): Rodrigues' formula (and the first-order branch below THETA2_SMALL)
    agrees with scipy's matrix exponential of the skew matrix at angles from 1e-9 to 3 rad, so
    the small-angle branch cannot be taken where its error would show."""
    import scipy.linalg as sla
    rng = np.random.default_rng(9)
    for th in (1e-9, 1e-7, 1e-5, 1e-3, 0.1, 1.0, 3.0):
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        w = th * k
        X = rng.normal(0, 5.0, size=3)
        K = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
        ref = sla.expm(K) @ X
        RX = np.array([v[0] for v in cm.rotate([np.array([wi]) for wi in w], [np.array([xi]) for xi in X])])
        np.testing.assert_allclose(RX, ref, rtol=0, atol=1e-14 * np.linalg.norm(X), err_msg=f"theta={th}")
