"""Shared helpers for the GPU parity tests: oracle references for a problem at its initial
state.  Imports only the oracle and the generator (never the CUDA path)."""
import numpy as np

from oracle import camera_model as cm
from oracle import normal_eq as neq
from oracle import power_series as ps


class OracleRef:
    """FP64 oracle quantities at (cams0, lms0) of a problem."""

    def __init__(self, p, cams=None, lms=None):
        self.p = p
        self.cams = p.cams0 if cams is None else cams
        self.lms = p.lms0 if lms is None else lms
        self.r, self.Jp, self.Jl = cm.linearize(self.cams, self.lms, p.obs, p.cam_idx, p.lm_idx, p.weights)
        self.ne = neq.NormalEquation(self.r, self.Jp, self.Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)

    def solve(self, lam, eps, m_max, damping_mode=0):
        Ul, Vl = self.ne.damped(lam, damping_mode)
        Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
        bt = neq.schur_rhs(self.ne, Vi)
        x, m, sv, hist = ps.power_series_solve(self.ne, Ui, Vi, bt, eps=eps, m_max=m_max)
        xl = neq.back_substitute(self.ne, Vi, x)
        return dict(x=x, xl=xl, m=m, sv=sv, bt=bt, Ul=Ul, Vi=Vi, hist=hist,
                    pred=neq.model_decrease(self.ne, x, xl))

    def schur_residual(self, lam, x, damping_mode=0):
        """||S x + b~|| / ||b~|| with S applied as U x - W V^-1 W^T x (matrix-free, oracle)."""
        Ul, Vl = self.ne.damped(lam, damping_mode)
        Vi = neq.chol_inverse(Vl)
        bt = neq.schur_rhs(self.ne, Vi)
        Sx = neq.apply_blocks(Ul, x) - self.ne.W @ neq.apply_blocks(Vi, self.ne.W.T @ x)
        return float(np.linalg.norm(Sx + bt) / np.linalg.norm(bt))


# per camera / landmark block (block_rel): an error confined to a few weakly observed blocks must
# not hide under the whole-vector norm.  Measured on the parity cases: FP64 at most 4e-11
# (bound 1e-8); FP32 bulk at most 1.1e-2 at lambda = 1e-4 (a two-view landmark, where float
# rounding of J is amplified by the conditioning of the series) and 9e-4 at lambda = 1e-2
# (bound 5e-2)
FP64_BLOCK_TOL = 1e-8
FP32_BLOCK_TOL = 5e-2


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def block_rel(a, b, width):
    """Largest per-block relative difference over the blocks of `width` values (a camera's 9 or a
    landmark's 3), each against its own norm, with a floor of 1e-6 of the largest block norm so
    that a block the step barely moves is not judged on its rounding alone."""
    a = np.asarray(a, dtype=np.float64).reshape(-1, width)
    b = np.asarray(b, dtype=np.float64).reshape(-1, width)
    nb = np.linalg.norm(b, axis=1)
    floor = 1e-6 * (nb.max() if nb.size and nb.max() > 0 else 1.0)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.maximum(nb, floor))) if nb.size else 0.0


def check_step_blocks(dxp, dxl, x_ref, xl_ref, precision):
    """Per-block bound of a step against the oracle's (cameras of 9, landmarks of 3)."""
    tol = FP64_BLOCK_TOL if precision == 0 else FP32_BLOCK_TOL
    bp, bl = block_rel(dxp, x_ref, 9), block_rel(dxl, xl_ref, 3)
    assert bp < tol and bl < tol, (precision, bp, bl)
