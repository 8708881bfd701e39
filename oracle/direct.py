"""Exact solves of the reduced camera system S dx_p = -b~ (FP64, CPU) -- test infrastructure only.

These are the references the truncated series of Sec. 4.3 converges to (Prop. 2):
  * dense Cholesky of the explicit S (Sec. 4.2 eq. `Schur`) for small camera counts;
  * conjugate gradients on the explicit block-sparse S with the Schur-Jacobi (9x9 block
    diagonal of S) preconditioner, the solver family the paper compares against (Sec. 5,
    "Ceres-explicit"), for large camera counts.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .normal_eq import NormalEquation, explicit_schur, block_diagonal, chol_inverse, apply_blocks

DENSE_LIMIT = 2000  # use the dense route when 9 n_c <= this


def solve_dense(S, b_tilde):
    """dx_p = -S^-1 b~ via Cholesky of the dense S."""
    c = sla.cho_factor(S, lower=True)
    return -sla.cho_solve(c, b_tilde)


def pcg(S, rhs, precond_blocks_inv, rtol=1e-12, max_iter=100000):
    """Preconditioned conjugate gradients (Hestenes-Stiefel) on S y = rhs.

    Returns (y, iterations, relative residual).
    """
    y = np.zeros_like(rhs)
    r = rhs.copy()
    bn = float(np.linalg.norm(rhs))
    if bn == 0.0:
        return y, 0, 0.0
    z = apply_blocks(precond_blocks_inv, r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    for it in range(1, max_iter + 1):
        Sp = S @ p
        alpha = rz / float(p @ Sp)
        y += alpha * p
        r -= alpha * Sp
        if float(np.linalg.norm(r)) <= rtol * bn:
            break
        z = apply_blocks(precond_blocks_inv, r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return y, it, float(np.linalg.norm(rhs - S @ y)) / bn


def solve_reduced(ne: NormalEquation, Ulam, Vinv, b_tilde, rtol=1e-12):
    """Exact dx_p of S dx_p = -b~: dense Cholesky when 9 n_c <= DENSE_LIMIT, else PCG."""
    if 9 * ne.n_cams <= DENSE_LIMIT:
        S = explicit_schur(ne, Ulam, Vinv, dense=True)
        return solve_dense(S, b_tilde)
    S = explicit_schur(ne, Ulam, Vinv, dense=False)
    Minv = chol_inverse(block_diagonal(S, ne.n_cams, 9))
    y, _, _ = pcg(S, -b_tilde, Minv, rtol=rtol)
    return y
