"""Preconditioned conjugate gradients on the reduced camera system (FP64, CPU) -- test
infrastructure only.

The comparison solvers around the paper's method.  Both solve S dx_p = -b~ (Sec. 4.2, eqs. `Sx`,
`Schur`) by conjugate gradients with S applied as U_lam t - W V_lam^-1 W^T t:
  * Schur-Jacobi preconditioning (Sec. 5: the preconditioner of Ceres-explicit and
    Ceres-implicit): M^-1 = the inverse of the 9x9 diagonal blocks of S,
    S_cc = U_lam,c - sum_l W_cl V_l^-1 W_cl^T;
  * power-series preconditioning (the Neumann-series preconditioner discussed with Fig. 2,
    "PoCG"): M^-1 = sum_{i=0..m} (U^-1 W V^-1 W^T)^i U^-1, i.e. the truncated series of eq.
    `S_approx` applied to the residual (each application costs m series terms).
CG is the Hestenes-Stiefel recursion; it stops when ||r|| <= rtol ||rhs|| or after max_iter
iterations.  The landmark step follows by back-substitution (Sec. 4.2).
"""
from __future__ import annotations

import numpy as np

from .normal_eq import (NormalEquation, apply_blocks, back_substitute, block_diagonal,
                        chol_inverse, explicit_schur, schur_rhs)
from .power_series import apply_P


def schur_apply(ne: NormalEquation, Ulam, Vinv, t):
    """S t = U_lam t - W V_lam^-1 W^T t (matrix-free)."""
    return apply_blocks(Ulam, t) - ne.W @ apply_blocks(Vinv, ne.W.T @ t)


def schur_jacobi_blocks(ne: NormalEquation, Ulam, Vinv):
    """The 9x9 diagonal blocks of S, from the explicit S (Sec. 4.2 eq. `Schur`)."""
    S = explicit_schur(ne, Ulam, Vinv, dense=False)
    return block_diagonal(S, ne.n_cams, 9)


def power_series_preconditioner(ne: NormalEquation, Uinv, Vinv, m):
    """r -> sum_{i=0..m} P^i U^-1 r with P = U^-1 W V^-1 W^T (eq. `S_approx`, m terms)."""
    def apply(r):
        t = apply_blocks(Uinv, r)
        z = t.copy()
        for _ in range(m):
            t = apply_P(ne, Uinv, Vinv, t)
            z = z + t
        return z
    return apply


def pcg(apply_S, rhs, apply_Minv, rtol=1e-10, max_iter=500):
    """Hestenes-Stiefel PCG on S y = rhs from y = 0.  Returns (y, iterations, ||r|| / ||rhs||)."""
    y = np.zeros_like(rhs)
    r = rhs.copy()
    bn = float(np.linalg.norm(rhs))
    if bn == 0.0:
        return y, 0, 0.0
    z = apply_Minv(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    rel = 1.0
    for it in range(1, max_iter + 1):
        q = apply_S(p)
        alpha = rz / float(p @ q)
        y = y + alpha * p
        r = r - alpha * q
        rel = float(np.linalg.norm(r)) / bn
        if rel <= rtol:
            break
        z = apply_Minv(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return y, it, rel


def pcg_solve(ne: NormalEquation, lam, precond="jacobi", m=2, rtol=1e-10, max_iter=500,
              damping_mode=0):
    """dx_p, dx_l of the damped normal equation by PCG on the reduced system (S y = -b~).
    precond: "jacobi" (Schur-Jacobi) or "power" (order-m series).  Returns
    (dx_p, dx_l, iterations, relative residual)."""
    Ul, Vl = ne.damped(lam, damping_mode)
    Vi = chol_inverse(Vl)
    bt = schur_rhs(ne, Vi)
    if precond == "jacobi":
        Mi = chol_inverse(schur_jacobi_blocks(ne, Ul, Vi))
        apply_Minv = lambda r: apply_blocks(Mi, r)
    elif precond == "power":
        apply_Minv = power_series_preconditioner(ne, chol_inverse(Ul), Vi, m)
    else:
        raise ValueError(precond)
    y, it, rel = pcg(lambda t: schur_apply(ne, Ul, Vi, t), -bt, apply_Minv, rtol, max_iter)
    return y, back_substitute(ne, Vi, y), it, rel
