"""Normal equation, damping, Schur complement and back-substitution (FP64, CPU) -- test
infrastructure only.

Sec. 4.1, eq. `normal`: H (dx_p; dx_l) = -(b_p; b_l) with
    H = [[U_lambda, W], [W^T, V_lambda]],  U_lambda = J_p^T J_p + lambda D_p^T D_p,
    V_lambda = J_l^T J_l + lambda D_l^T D_l,  W = J_p^T J_l,  b_p = J_p^T r,  b_l = J_l^T r.
Sec. 4.2, eqs. `Sx`, `Schur`: S dx_p = -b~,  S = U_lambda - W V_lambda^-1 W^T,
    b~ = b_p - W V_lambda^-1 b_l.
Sec. 4.2, eq. `back_substitution`: the paper prints dx_l = -V^-1(-b_l + W^T dx_p); the second
block row of the normal equation gives dx_l = -V_lambda^-1 (b_l + W^T dx_p), which is used.

The damping matrices D_p, D_l are not defined in the paper.  Reading (Marquardt / Ceres style,
consistent with "in line with [rootba] and Ceres", Sec. 5.1): D^T D = diag(J^T J) clamped to
[DAMP_MIN, DAMP_MAX] (damping_mode 0), or D = I (damping_mode 1).

Everything here is the plain definition: the sparse Jacobian is assembled from the per-
observation blocks and the products J^T J, J^T r are formed with scipy.sparse.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DAMP_MIN = 1e-6
DAMP_MAX = 1e32


def assemble_jacobians(Jp, Jl, cam_idx, lm_idx, n_cams, n_lms):
    """Sparse J_p [2 n_o, 9 n_c] and J_l [2 n_o, 3 n_l] from per-observation blocks."""
    n = Jp.shape[0]
    o = np.arange(n)
    rows_p = (2 * o[:, None, None] + np.arange(2)[None, :, None]) + np.zeros((1, 1, 9), dtype=np.int64)
    cols_p = (9 * cam_idx.astype(np.int64)[:, None, None] + np.arange(9)[None, None, :]) + np.zeros((1, 2, 1), dtype=np.int64)
    Jps = sp.csr_matrix((Jp.ravel(), (rows_p.ravel(), cols_p.ravel())), shape=(2 * n, 9 * n_cams))
    rows_l = (2 * o[:, None, None] + np.arange(2)[None, :, None]) + np.zeros((1, 1, 3), dtype=np.int64)
    cols_l = (3 * lm_idx.astype(np.int64)[:, None, None] + np.arange(3)[None, None, :]) + np.zeros((1, 2, 1), dtype=np.int64)
    Jls = sp.csr_matrix((Jl.ravel(), (rows_l.ravel(), cols_l.ravel())), shape=(2 * n, 3 * n_lms))
    return Jps, Jls


def block_diagonal(M, n_blocks, d):
    """Dense [n_blocks, d, d] copy of the diagonal d x d blocks of a sparse matrix."""
    C = M.tocoo()
    keep = (C.row // d) == (C.col // d)
    out = np.zeros((n_blocks, d, d))
    np.add.at(out, (C.row[keep] // d, C.row[keep] % d, C.col[keep] % d), C.data[keep])
    return out


def _bd_fast(blocks):
    """Sparse CSR block-diagonal matrix from dense blocks [n, d, d]."""
    n, d, _ = blocks.shape
    b = np.arange(n)[:, None, None]
    rows = d * b + np.arange(d)[None, :, None] + np.zeros((1, 1, d), dtype=np.int64)
    cols = d * b + np.arange(d)[None, None, :] + np.zeros((1, d, 1), dtype=np.int64)
    return sp.csr_matrix((blocks.ravel(), (rows.ravel(), cols.ravel())), shape=(n * d, n * d))


class NormalEquation:
    """Undamped blocks of eq. `normal` at one linearisation point (r, J_p, J_l)."""

    def __init__(self, r, Jp, Jl, cam_idx, lm_idx, n_cams, n_lms):
        self.n_cams, self.n_lms = n_cams, n_lms
        self.r = r
        self.Jps, self.Jls = assemble_jacobians(Jp, Jl, cam_idx, lm_idx, n_cams, n_lms)
        rv = r.ravel()
        Up = (self.Jps.T @ self.Jps).tocsr()           # J_p^T J_p
        Vl = (self.Jls.T @ self.Jls).tocsr()           # J_l^T J_l
        self.U = block_diagonal(Up, n_cams, 9)         # [n_c, 9, 9]
        self.V = block_diagonal(Vl, n_lms, 3)          # [n_l, 3, 3]
        self.W = (self.Jps.T @ self.Jls).tocsr()       # [9 n_c, 3 n_l]
        self.b_p = self.Jps.T @ rv                     # [9 n_c]
        self.b_l = self.Jls.T @ rv                     # [3 n_l]

    def damped(self, lam, damping_mode=0):
        """(U_lambda, V_lambda) block arrays for the damping reading stated above."""
        return damp(self.U, lam, damping_mode), damp(self.V, lam, damping_mode)


def damp(blocks, lam, damping_mode=0):
    """blocks + lambda D^T D with D^T D = clamp(diag(blocks)) (mode 0) or I (mode 1)."""
    out = blocks.copy()
    d = blocks.shape[1]
    idx = np.arange(d)
    if damping_mode == 0:
        diag = np.clip(blocks[:, idx, idx], DAMP_MIN, DAMP_MAX)
    else:
        diag = np.ones((blocks.shape[0], d))
    out[:, idx, idx] += lam * diag
    return out


def chol_inverse(blocks):
    """Inverse of each SPD block via its Cholesky factor L: A^-1 = L^-T L^-1.

    Raises numpy.linalg.LinAlgError when a block is not positive definite (Sec. 4.1 states
    U_lambda and V_lambda are SPD).
    """
    L = np.linalg.cholesky(blocks)
    Li = np.linalg.inv(L)
    return np.einsum("nji,njk->nik", Li, Li)


def apply_blocks(blocks, v):
    """Block-diagonal matrix-vector product; v has length n * d."""
    n, d, _ = blocks.shape
    return np.einsum("nij,nj->ni", blocks, v.reshape(n, d)).ravel()


def schur_rhs(ne: NormalEquation, Vinv):
    """b~ = b_p - W V_lambda^-1 b_l (Sec. 4.2)."""
    return ne.b_p - ne.W @ apply_blocks(Vinv, ne.b_l)


def explicit_schur(ne: NormalEquation, Ulam, Vinv, dense=True):
    """S = U_lambda - W V_lambda^-1 W^T (Sec. 4.2 eq. `Schur`), dense or sparse CSR."""
    Vi = _bd_fast(Vinv)
    WVW = (ne.W @ Vi @ ne.W.T).tocsr()
    S = _bd_fast(Ulam) - WVW
    return S.toarray() if dense else S.tocsr()


def back_substitute(ne: NormalEquation, Vinv, dx_p):
    """dx_l = -V_lambda^-1 (b_l + W^T dx_p) (Sec. 4.2, sign derived from eq. `normal`)."""
    return -apply_blocks(Vinv, ne.b_l + ne.W.T @ dx_p)


def model_decrease(ne: NormalEquation, dx_p, dx_l):
    """L(0) - L(dx) = 1/2 ||r||^2 - 1/2 ||r + J_p dx_p + J_l dx_l||^2 (undamped model)."""
    rv = ne.r.ravel()
    rn = rv + ne.Jps @ dx_p + ne.Jls @ dx_l
    return 0.5 * float(rv @ rv) - 0.5 * float(rn @ rn)
