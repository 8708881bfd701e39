"""Pins for the oracle's power series (Sec. 4.3, Lemma 1, Prop. 1, Prop. 2, eq. `qcriterion`).

P = U^-1 W V^-1 W^T is not symmetric, so the norm bounds are checked in the U-weighted norm
||e||_U = ||U^(1/2) e||_2, in which P is self-adjoint and ||P||_U = rho(P)."""
import numpy as np
import pytest
import scipy.linalg as sla

import bal_synth
from oracle import camera_model as cm
from oracle import normal_eq as neq
from oracle import power_series as ps
from oracle import direct


def _setup(lam=1e-4, seed=31, nc=5, nl=60):
    p = bal_synth.make_problem(nc, nl, track=("uniform", 2, 4), seed=seed)
    r, Jp, Jl = cm.linearize(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    Ul, Vl = ne.damped(lam)
    Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
    bt = neq.schur_rhs(ne, Vi)
    # dense operators, formed independently of the oracle's recursion
    Ud = sla.block_diag(*Ul)
    Uid = np.linalg.inv(Ud)
    Vid = np.linalg.inv(sla.block_diag(*Vl))
    Wd = ne.W.toarray()
    P = Uid @ Wd @ Vid @ Wd.T
    S = Ud - Wd @ Vid @ Wd.T
    dx_exact = np.linalg.solve(S, -bt)
    return ne, Ui, Vi, bt, Ud, P, S, dx_exact


@pytest.mark.parametrize("lam", [1e-4, 1e-1, 10.0])
def test_lemma1_eigenvalues_in_unit_interval(lam):
    _, _, _, _, _, P, _, _ = _setup(lam)
    ev = np.linalg.eigvals(P)
    assert np.abs(ev.imag).max() < 1e-8
    assert ev.real.min() > -1e-10
    assert ev.real.max() < 1.0


def test_factorisation_S_equals_U_times_I_minus_P():
    _, _, _, _, Ud, P, S, _ = _setup()
    np.testing.assert_allclose(Ud @ (np.eye(P.shape[0]) - P), S, rtol=0, atol=1e-8 * np.abs(S).max())


@pytest.mark.parametrize("m", [0, 1, 2, 5, 12])
def test_truncation_error_identity(m):
    """x(m) - dx_p = -P^(m+1) dx_p, which follows from R_m = sum_{i>m} P^i U^-1 (Prop. 2)."""
    ne, Ui, Vi, bt, Ud, P, S, dx = _setup(lam=1e-2)
    x, mm, _, _ = ps.power_series_solve(ne, Ui, Vi, bt, eps=0.0, m_max=m)
    assert mm == m
    ref = dx - np.linalg.matrix_power(P, m + 1) @ dx
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-9


def test_error_bound_in_U_norm_and_prop1_equality():
    ne, Ui, Vi, bt, Ud, P, S, dx = _setup(lam=1e-2)
    Uh = sla.sqrtm(Ud).real
    Uhi = np.linalg.inv(Uh)
    rho = max(np.linalg.eigvals(P).real)
    unorm = lambda e: np.linalg.norm(Uh @ e)
    prev = np.inf
    for m in range(0, 15):
        x, _, _, _ = ps.power_series_solve(ne, Ui, Vi, bt, eps=0.0, m_max=m)
        err = unorm(x - dx)
        assert err <= rho ** (m + 1) * unorm(dx) * (1 + 1e-8) + 1e-14
        assert err <= prev * (1 + 1e-10)  # monotone in the U-norm
        prev = err
        # Prop. 1: ||R|| <= ||P||^(m+1) / (1 - ||P||) with R = P^(m+1) (I - P)^-1; in the
        # U-norm all eigenvalues are in [0, 1), so the bound holds with equality.
        R = np.linalg.matrix_power(P, m + 1) @ np.linalg.inv(np.eye(P.shape[0]) - P)
        Rn = np.linalg.norm(Uh @ R @ Uhi, 2)
        bound = rho ** (m + 1) / (1 - rho)
        assert Rn <= bound * (1 + 1e-6)
        assert Rn >= bound * (1 - 1e-6)


def test_series_converges_to_exact_solve_at_large_lambda():
    ne, Ui, Vi, bt, Ud, P, S, dx = _setup(lam=10.0)
    x, m, sv, _ = ps.power_series_solve(ne, Ui, Vi, bt, eps=1e-14, m_max=400)
    assert np.linalg.norm(x - dx) / np.linalg.norm(dx) < 1e-10


def test_stop_index_matches_dense_partial_sums():
    """The stop index of the recursion equals the first i with (i+1)||x(i)-x(i-1)||/||x(i)||
    < eps where x(i) = -sum_{j<=i} P^j U^-1 b~ is formed with dense matrix powers."""
    for eps in (0.5, 0.1, 0.03):
        ne, Ui, Vi, bt, Ud, P, S, dx = _setup(lam=1.0)
        x, m, sv, hist = ps.power_series_solve(ne, Ui, Vi, bt, eps=eps, m_max=20)
        u = -np.linalg.solve(Ud, bt)
        xs = [u]
        term = u
        for i in range(1, 21):
            term = P @ term
            xs.append(xs[-1] + term)
        expect = 20
        for i in range(1, 21):
            if (i + 1) * np.linalg.norm(xs[i] - xs[i - 1]) / np.linalg.norm(xs[i]) < eps:
                expect = i
                break
        assert m == expect, (eps, m, expect)
        assert np.linalg.norm(x - xs[expect]) / np.linalg.norm(xs[expect]) < 1e-12
        # the returned stop value is the left-hand side of eq. `qcriterion` at the stop index
        sv_ref = (expect + 1) * np.linalg.norm(xs[expect] - xs[expect - 1]) / np.linalg.norm(xs[expect])
        assert abs(sv - sv_ref) <= 1e-9 * sv_ref, (eps, sv, sv_ref)


def test_stop_rule_scripted_sequences():
    # (i + 1) * ||t_i|| / ||x(i)|| < eps, i >= 1
    x = [1.0] * 6
    assert ps.run_stop_rule([9, 1.0, 0.1, 0.001, 0, 0], x, 0.01, 20) == 3  # 2.0, 0.3, 0.004
    assert ps.run_stop_rule([9, 0.004, 1, 1, 1, 1], x, 0.01, 20) == 1      # 2 * 0.004 = 0.008
    assert ps.run_stop_rule([9, 0.005, 1, 1, 1, 1], x, 0.01, 5) == 5       # 0.010 is not < 0.01
    assert ps.run_stop_rule([9, 1, 1, 1, 1, 1], [1, 1, 0.0, 1, 1, 1], 0.01, 5) == 2  # ||x|| = 0
    # the test starts at i = 1: a small ratio at i = 0 (1 * 0.001) does not stop the series
    assert ps.run_stop_rule([0.001, 1, 0.001, 1, 1, 1], x, 0.01, 20) == 2  # 2.0, 0.003
    assert ps.stop_test(3, 0.0024, 1.0, 0.01)                                # 4 * 0.0024 = 0.0096
    assert not ps.stop_test(3, 0.0025, 1.0, 0.01)                            # 0.0100


def test_zero_rhs_returns_zero():
    ne, Ui, Vi, bt, *_ = _setup()
    x, m, sv, _ = ps.power_series_solve(ne, Ui, Vi, np.zeros_like(bt), eps=0.01, m_max=20)
    assert m == 0 and np.all(x == 0)
