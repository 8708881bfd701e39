"""Power-series solve of the reduced camera system (FP64, CPU) -- test infrastructure only.

Sec. 4.3: S = U_lambda (I - P) with P = U_lambda^-1 W V_lambda^-1 W^T (eq. `inverse`), so
S^-1 = (I - P)^-1 U_lambda^-1.  Lemma 1 puts every eigenvalue of P in [0, 1), so the Neumann
series of Prop. 1 applies and the truncated inverse is (eq. `S_approx`)

    S~_-1(m) = sum_{i=0}^{m} P^i U_lambda^-1,       x(m) = -S~_-1(m) b~     (eq. `x_approx`).

The terms are generated by recursion, t_0 = x(0) = -U^-1 b~, t_i = P t_{i-1},
x(i) = x(i-1) + t_i, so that x(i) - x(i-1) = t_i.

Stop rule (eq. `qcriterion`, Sec. 4.3): stop at the first i >= 1 with
    (i + 1) ||x(i) - x(i-1)||_2 / ||x(i)||_2 < eps,
with eps = 0.01 and at most 20 inner iterations (Sec. 5.1).  Readings: the test starts at i = 1
(x(-1) does not exist); "20 inner iterations" means at most 20 applications of P, i.e. terms
x(0) .. x(20); the returned vector is the x(i) at which the test fired (or x(m_max)); if
||x(i)|| = 0 the zero vector is returned.
"""
from __future__ import annotations

import numpy as np

from .normal_eq import NormalEquation, apply_blocks


def stop_test(i, t_norm, x_norm, eps):
    """The eq. `qcriterion` test at inner iteration i (True = stop)."""
    if x_norm == 0.0:
        return True
    return (i + 1) * t_norm / x_norm < eps


def apply_P(ne: NormalEquation, Uinv, Vinv, t):
    """P t = U^-1 (W (V^-1 (W^T t))) (Sec. 4.3, the operator of eq. `inverse`)."""
    return apply_blocks(Uinv, ne.W @ apply_blocks(Vinv, ne.W.T @ t))


def power_series_solve(ne: NormalEquation, Uinv, Vinv, b_tilde, eps=0.01, m_max=20):
    """x(m) of eq. `x_approx` with the stop rule of eq. `qcriterion`.

    Returns (x, m, stop_value, history) where m is the number of P applications performed and
    history lists (i, ||t_i||, ||x(i)||) for i = 0..m.
    """
    t = -apply_blocks(Uinv, b_tilde)
    x = t.copy()
    xn = float(np.linalg.norm(x))
    history = [(0, xn, xn)]
    if xn == 0.0:
        return np.zeros_like(x), 0, 0.0, history
    stop_value = float("inf")
    m = 0
    for i in range(1, m_max + 1):
        t = apply_P(ne, Uinv, Vinv, t)
        x = x + t
        m = i
        tn = float(np.linalg.norm(t))
        xn = float(np.linalg.norm(x))
        history.append((i, tn, xn))
        if xn == 0.0:
            return np.zeros_like(x), m, 0.0, history
        stop_value = (i + 1) * tn / xn
        if stop_value < eps:
            break
    return x, m, stop_value, history


def run_stop_rule(term_norms, x_norms, eps, m_max):
    """Stop index for scripted norm sequences (i = 1..): first i with the test true, else m_max."""
    for i in range(1, m_max + 1):
        if stop_test(i, term_norms[i], x_norms[i], eps):
            return i
    return m_max
