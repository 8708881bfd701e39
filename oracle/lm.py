"""Levenberg-Marquardt outer loop (FP64, CPU) -- test infrastructure only.

Sec. 5.1 ("LM loop"): start with damping 1e-4, update lambda on success or failure, at most 50
LM iterations, stop early at a relative function tolerance of 1e-6; at most 20 inner (series)
iterations with eps = 0.01.  Each iteration linearises (Sec. 4.1), damps and inverts the
blocks, solves the reduced camera system (Sec. 4.3 power series, or an exact solve for
reference), back-substitutes (Sec. 4.2) and evaluates the new cost (Sec. 4).

The paper does not print the lambda update.  Reading (Nielsen-type rule of the Ceres / rootba
family): gain ratio rho = (F(x) - F(x + dx)) / (L(0) - L(dx)) with the model decrease computed
directly from r and J; the step is accepted iff F decreased and L(0) - L(dx) > 0; on accept
lambda <- lambda max(1/3, 1 - (2 rho - 1)^3), nu <- 2; on reject lambda <- lambda nu,
nu <- 2 nu; lambda is clamped to [1e-10, 1e32].  Rejected steps re-solve with the new lambda at
the same linearisation.  Sec. 4.1 takes the damped blocks to be positive definite; in floating
point a block can still fail its Cholesky factorisation (lambda so small that the damping
underflows, or a nearly singular block).  Reading: such an iteration has no step -- it is
rejected like a step that did not decrease F (state unchanged, lambda <- lambda nu), and its
history entry has not_spd = True and cost_after = NaN.  The run stops after an accepted step
whose relative decrease (F_old - F_new) / F_old is below func_tol, or after max_lm iterations.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import camera_model as cm
from .normal_eq import NormalEquation, chol_inverse, schur_rhs, back_substitute, model_decrease
from .power_series import power_series_solve
from .direct import solve_reduced

LAMBDA_MIN = 1e-10
LAMBDA_MAX = 1e32


@dataclasses.dataclass
class Options:
    """The LM and series settings; the defaults are those of Sec. 5.1."""
    lambda0: float = 1e-4
    func_tol: float = 1e-6
    eps: float = 0.01
    max_lm: int = 50
    max_inner: int = 20
    damping_mode: int = 0


def lambda_update(lam, nu, accepted, rho):
    """Next (lambda, nu) for the reading stated in the module docstring."""
    if accepted:
        lam = lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
        nu = 2.0
    else:
        lam = lam * nu
        nu = 2.0 * nu
    return min(max(lam, LAMBDA_MIN), LAMBDA_MAX), nu


def solve_step(ne: NormalEquation, lam, opts: Options, solver="power"):
    """One damped solve: returns dx_p, dx_l and series info (m, stop value)."""
    Ulam, Vlam = ne.damped(lam, opts.damping_mode)
    Uinv, Vinv = chol_inverse(Ulam), chol_inverse(Vlam)
    bt = schur_rhs(ne, Vinv)
    if solver == "power":
        dx_p, m, sv, _ = power_series_solve(ne, Uinv, Vinv, bt, opts.eps, opts.max_inner)
    else:
        dx_p, m, sv = solve_reduced(ne, Ulam, Vinv, bt), -1, 0.0
    dx_l = back_substitute(ne, Vinv, dx_p)
    return dx_p, dx_l, m, sv


def lm_solve(problem, opts: Options | None = None, solver="power", cams=None, lms=None):
    """Run LM from the problem's initial state.  Returns (cams, lms, history)."""
    opts = opts or Options()
    cams = (problem.cams0 if cams is None else cams).copy()
    lms = (problem.lms0 if lms is None else lms).copy()
    args = (problem.obs, problem.cam_idx, problem.lm_idx, problem.weights)
    nc, nl = cams.shape[0], lms.shape[0]
    lam, nu = opts.lambda0, 2.0
    F = cm.cost(cams, lms, *args)
    ne = None
    history = []
    for it in range(opts.max_lm):
        if ne is None:
            r, Jp, Jl = cm.linearize(cams, lms, *args)
            ne = NormalEquation(r, Jp, Jl, problem.cam_idx, problem.lm_idx, nc, nl)
        try:
            dx_p, dx_l, m, sv = solve_step(ne, lam, opts, solver)
        except np.linalg.LinAlgError:
            history.append(dict(it=it, cost_before=F, cost_after=np.nan, lam=lam, accepted=False,
                                rho=0.0, inner=0, stop_value=np.inf, pred=0.0, not_spd=True))
            lam, nu = lambda_update(lam, nu, False, 0.0)
            continue
        cams_new = cams + dx_p.reshape(nc, 9)
        lms_new = lms + dx_l.reshape(nl, 3)
        F_new = cm.cost(cams_new, lms_new, *args)
        pred = model_decrease(ne, dx_p, dx_l)
        actual = F - F_new
        accepted = bool(np.isfinite(F_new) and actual > 0.0 and pred > 0.0)
        rho = actual / pred if pred != 0.0 else 0.0
        history.append(dict(it=it, cost_before=F, cost_after=F_new, lam=lam, accepted=accepted,
                            rho=rho, inner=m, stop_value=sv, pred=pred, not_spd=False))
        lam, nu = lambda_update(lam, nu, accepted, rho)
        if accepted:
            cams, lms = cams_new, lms_new
            F_old, F = F, F_new
            ne = None
            if (F_old - F_new) / F_old < opts.func_tol:
                break
    return cams, lms, history
