"""Implicit-differentiation adjoint of the bundle-adjustment solution (FP64, CPU) -- test
infrastructure only.

The paper has no adjoint; this is the differentiable form built around its solver.  Reading:
the solution x* minimises F(x; obs, w) = 1/2 sum_o w_o ||pi_o(x) - obs_o||^2 (Sec. 4), so it
satisfies g(x*, theta) = sum_o w_o J_o^T r_o = 0 with theta = (obs, w), r_o = pi_o(x) - obs_o
and J_o = d pi_o / dx.  By the implicit-function theorem dx*/dtheta = -(dg/dx)^-1 dg/dtheta.
The damped Gauss-Newton matrix of eq. `normal`, H_lam = J^T W J + lam D^T D (the same damping
as the LM step), stands in for dg/dx: it is what the solver inverts, and the damping removes the
7-dimensional gauge freedom (rotation, translation, scale) that makes J^T W J singular.  For a
scalar L(x*) with incoming gradient (g_p, g_l) = dL/dx*, the adjoint vector is

    a = H_lam^-1 (g_p; g_l),

solved like a step of eq. `normal` with the right-hand side -(g_p; g_l): the reduced system
S a_p = g_p - W V_lam^-1 g_l (Sec. 4.2) and a_l = V_lam^-1 (g_l - W^T a_p).  Then, with a_o the
part of a belonging to observation o's camera and landmark,

    dL/dobs_o = -(dg/dobs_o)^T a = w_o J_o a_o,
    dL/dw_o   = -(dg/dw_o)^T a   = -r_o^T J_o a_o.

For a damped Gauss-Newton step taken at a fixed linearisation point, dx = -H_lam^-1 J^T W r, the
first formula is the exact derivative of g^T dx with respect to obs (r is linear in obs, H_lam
and J do not depend on it), and at a point where J^T W r = 0 the second one is the exact
derivative with respect to w.  At a minimiser of F plus the prior lam/2 ||D (x - x0)||^2 with
x0 = x*, both are exact up to the second-order residual terms sum_o w_o r_o d^2 r_o that Gauss-
Newton drops (zero when the residuals are zero).  tests/test_oracle_adjoint.py checks each of
these statements against finite differences.
"""
from __future__ import annotations

import numpy as np

from . import camera_model as cm
from .direct import solve_reduced
from .normal_eq import NormalEquation, apply_blocks, chol_inverse
from .power_series import power_series_solve


def adjoint_solve(ne: NormalEquation, lam, g_p, g_l, damping_mode=0, solver="direct", eps=0.0,
                  m_max=20):
    """a = H_lam^-1 (g_p; g_l) through the Schur complement.  solver "direct": the exact reduced
    solve; "power": the truncated series of Sec. 4.3 (eq. `x_approx`) with the stop rule of eq.
    `qcriterion` (eps, m_max).  Returns (a_p, a_l, m) with m = -1 for the direct solve."""
    Ul, Vl = ne.damped(lam, damping_mode)
    Vi = chol_inverse(Vl)
    rhs = g_p - ne.W @ apply_blocks(Vi, g_l)  # S a_p = rhs, i.e. b~ = -rhs in eq. `Sx`
    if solver == "direct":
        a_p = solve_reduced(ne, Ul, Vi, -rhs)
        m = -1
    else:
        Ui = chol_inverse(Ul)
        a_p, m, _, _ = power_series_solve(ne, Ui, Vi, -rhs, eps=eps, m_max=m_max)
    a_l = apply_blocks(Vi, g_l - ne.W.T @ a_p)
    return a_p, a_l, m


def observation_gradients(r, Jp, Jl, weights, cam_idx, lm_idx, a_p, a_l):
    """(dL/dobs [n_o, 2], dL/dw [n_o]) from the adjoint vector.  r, Jp, Jl are the weighted
    quantities sqrt(w) r, sqrt(w) J of camera_model.linearize, so w J a = sqrt(w) (sqrt(w) J) a
    and r^T J a = (sqrt(w) r)^T (sqrt(w) J) a / w."""
    ap = a_p.reshape(-1, 9)[cam_idx]
    al = a_l.reshape(-1, 3)[lm_idx]
    u = np.einsum("oij,oj->oi", Jp, ap) + np.einsum("oij,oj->oi", Jl, al)  # sqrt(w) J_o a_o
    w = np.ones(r.shape[0]) if weights is None else np.asarray(weights, dtype=np.float64)
    d_obs = np.sqrt(w)[:, None] * u
    d_w = -np.sum(r * u, axis=1) / w
    return d_obs, d_w


def gradients(problem, cams, lms, g_cams, g_lms, lam, damping_mode=0, solver="direct", eps=0.0,
              m_max=20):
    """dL/dobs and dL/dw at the state (cams, lms) for the incoming gradients g_cams [n_c, 9],
    g_lms [n_l, 3].  Returns (d_obs, d_w, a_p, a_l, m)."""
    p = problem
    r, Jp, Jl = cm.linearize(cams, lms, p.obs, p.cam_idx, p.lm_idx, p.weights)
    ne = NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, cams.shape[0], lms.shape[0])
    a_p, a_l, m = adjoint_solve(ne, lam, np.ravel(g_cams), np.ravel(g_lms), damping_mode,
                                solver, eps, m_max)
    d_obs, d_w = observation_gradients(r, Jp, Jl, p.weights, p.cam_idx, p.lm_idx, a_p, a_l)
    return d_obs, d_w, a_p, a_l, m
