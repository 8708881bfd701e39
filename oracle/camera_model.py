"""BAL camera model, residuals and Jacobians (FP64, CPU) -- test infrastructure only.

Sec. 4: the objective is F(x) = 1/2 sum_i ||r_i(x)||^2 over all observations, with state
x = (x_p, x_l), d_p = 9 camera parameters (rotation, translation and intrinsics) and 3 landmark
coordinates.  The paper does not print the projection; it uses the BAL convention (ref. [1],
"Bundle adjustment in the large"):

    P = R(w) X + t,   p = -P_xy / P_z,   pi = f (1 + k1 |p|^2 + k2 |p|^4) p,   r = pi - obs

with R(w) from Rodrigues' formula (vector form) and the first-order form X + w x X when
|w|^2 < THETA2_SMALL.  Observation weights w_o (not in the paper) enter as sqrt(w_o) r_o so that
F = 1/2 sum_o w_o ||r_o||^2.

Jacobians J_p = dr/dx_p (2x9) and J_l = dr/dx_l (2x3) come from forward-mode dual numbers pushed
through the same expression -- no hand-derived chain rule -- so they are an independent
derivation from any analytic Jacobian.
"""
from __future__ import annotations

import numpy as np

# First-order rotation branch below this |w|^2 (double machine epsilon).
THETA2_SMALL = float(np.finfo(np.float64).eps)


class Dual:
    """Value v [n] with gradient d [n, K] (forward-mode automatic differentiation)."""

    __slots__ = ("v", "d")

    def __init__(self, v, d):
        self.v = v
        self.d = d

    @staticmethod
    def _split(o):
        if isinstance(o, Dual):
            return o.v, o.d
        return o, None

    def __add__(self, o):
        ov, od = Dual._split(o)
        return Dual(self.v + ov, self.d if od is None else self.d + od)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        ov, od = Dual._split(o)
        return Dual(self.v - ov, self.d if od is None else self.d - od)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        ov, od = Dual._split(o)
        if od is None:
            return Dual(self.v * ov, self.d * np.asarray(ov)[..., None])
        return Dual(self.v * ov, self.d * ov[..., None] + od * self.v[..., None])

    __rmul__ = __mul__

    def __truediv__(self, o):
        ov, od = Dual._split(o)
        if od is None:
            return Dual(self.v / ov, self.d / np.asarray(ov)[..., None])
        q = self.v / ov
        return Dual(q, (self.d - od * q[..., None]) / ov[..., None])

    def __rtruediv__(self, o):
        # o / self with o a plain array
        q = o / self.v
        return Dual(q, -self.d * (q / self.v)[..., None])


def _sin(x):
    """sin of an array or Dual (derivative cos x)."""
    if isinstance(x, Dual):
        return Dual(np.sin(x.v), x.d * np.cos(x.v)[..., None])
    return np.sin(x)


def _cos(x):
    """cos of an array or Dual (derivative -sin x)."""
    if isinstance(x, Dual):
        return Dual(np.cos(x.v), -x.d * np.sin(x.v)[..., None])
    return np.cos(x)


def _sqrt(x):
    """sqrt of an array or Dual (derivative 1 / (2 sqrt x))."""
    if isinstance(x, Dual):
        s = np.sqrt(x.v)
        return Dual(s, x.d * (0.5 / s)[..., None])
    return np.sqrt(x)


def _where(mask, a, b):
    """Element-wise select between two (Dual or array) values."""
    if isinstance(a, Dual) or isinstance(b, Dual):
        av, ad = (a.v, a.d) if isinstance(a, Dual) else (a, np.zeros_like(b.d))
        bv, bd = (b.v, b.d) if isinstance(b, Dual) else (b, np.zeros_like(a.d))
        return Dual(np.where(mask, av, bv), np.where(mask[..., None], ad, bd))
    return np.where(mask, a, b)


def _value(x):
    """The value part of a Dual, or the array itself."""
    return x.v if isinstance(x, Dual) else x


def _cross(a, b):
    """Cross product a x b of two 3-component lists (arrays or Duals)."""
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def rotate(w, X):
    """R(w) X by Rodrigues' formula: X cos th + (k x X) sin th + k (k.X)(1 - cos th), k = w/th.

    w and X are lists of 3 components (arrays or Duals).  For th^2 < THETA2_SMALL the
    first-order form X + w x X is used.
    """
    th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2]
    small = _value(th2) < THETA2_SMALL
    # Evaluate the full formula on a safe angle where the first-order branch is taken.
    th2_safe = _where(small, np.ones_like(_value(th2)), th2)
    th = _sqrt(th2_safe)
    c, s = _cos(th), _sin(th)
    k = [w[i] / th for i in range(3)]
    kxX = _cross(k, X)
    kdX = k[0] * X[0] + k[1] * X[1] + k[2] * X[2]
    full = [X[i] * c + kxX[i] * s + k[i] * kdX * (1.0 - c) for i in range(3)]
    wxX = _cross(w, X)
    first = [X[i] + wxX[i] for i in range(3)]
    return [_where(small, first[i], full[i]) for i in range(3)]


def project(cam, X):
    """BAL projection pi(cam, X) for cam = [w0,w1,w2,t0,t1,t2,f,k1,k2] and landmark X."""
    RX = rotate(cam[0:3], X)
    P = [RX[i] + cam[3 + i] for i in range(3)]
    px = -P[0] / P[2]
    py = -P[1] / P[2]
    n2 = px * px + py * py
    rad = 1.0 + cam[7] * n2 + cam[8] * n2 * n2
    return [cam[6] * rad * px, cam[6] * rad * py]


def residuals(cams, lms, obs, cam_idx, lm_idx, weights=None):
    """r [n_o, 2] = sqrt(w) (pi(cam_c(o), X_l(o)) - obs_o), FP64."""
    c = cams[cam_idx]
    X = lms[lm_idx]
    pi = project([c[:, j] for j in range(9)], [X[:, j] for j in range(3)])
    r = np.stack([pi[0] - obs[:, 0], pi[1] - obs[:, 1]], axis=1)
    if weights is not None:
        r = r * np.sqrt(weights)[:, None]
    return r


def cost(cams, lms, obs, cam_idx, lm_idx, weights=None):
    """F(x) = 1/2 sum_o ||r_o||^2 (Sec. 4)."""
    r = residuals(cams, lms, obs, cam_idx, lm_idx, weights)
    return 0.5 * float(np.sum(r * r))


def linearize(cams, lms, obs, cam_idx, lm_idx, weights=None):
    """Residuals r [n_o,2], J_p [n_o,2,9], J_l [n_o,2,3] at the given state (Sec. 4.1).

    The 12 inputs of each observation (9 camera, 3 landmark) are seeded as dual directions.
    """
    n = obs.shape[0]
    c = cams[cam_idx]
    X = lms[lm_idx]
    eye = np.eye(12)
    cam = [Dual(c[:, j], np.broadcast_to(eye[j], (n, 12))) for j in range(9)]
    lm = [Dual(X[:, j], np.broadcast_to(eye[9 + j], (n, 12))) for j in range(3)]
    pi = project(cam, lm)
    r = np.stack([pi[0].v - obs[:, 0], pi[1].v - obs[:, 1]], axis=1)
    J = np.stack([pi[0].d, pi[1].d], axis=1)  # [n, 2, 12]
    if weights is not None:
        sw = np.sqrt(weights)
        r = r * sw[:, None]
        J = J * sw[:, None, None]
    return r, np.ascontiguousarray(J[:, :, 0:9]), np.ascontiguousarray(J[:, :, 9:12])
