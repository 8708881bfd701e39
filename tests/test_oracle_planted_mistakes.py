"""Planted mistakes in the oracle (CPU only).

Each case below makes one small edit to one oracle function in memory: a dropped term or line,
a flipped sign, a swapped index or operand, an off-by-one bound, a wrong update rule.  The
edited function is compiled in its module's namespace and put in place of the original (also in
every oracle or pin module that imported it by name); then the pins named for the case run.
The case passes when every one of those pins fails with an AssertionError.

This shows that the pins of tests/test_oracle_*.py constrain each part of the oracle (camera
model, Jacobians, normal equation, damping, inverses, Schur complement, back-substitution,
power series, stop rule, exact solves, PCG, LM loop, adjoint) through facts fixed by the paper,
the mathematics or a stated reading of the paper, not by re-running the oracle against itself.

An edit whose text no longer occurs exactly once in the oracle fails loudly, so a later change
to the oracle cannot turn a case into a silent no-op.  A control test runs every pin used here
without an edit and requires it to pass.
"""
import __future__
import inspect
import textwrap
from dataclasses import dataclass

import numpy as np
import pytest

from oracle import adjoint as o_adj
from oracle import camera_model as o_cm
from oracle import direct as o_direct
from oracle import lm as o_lm
from oracle import normal_eq as o_neq
from oracle import pcg as o_pcg
from oracle import power_series as o_ps

import test_oracle_adjoint as pin_adj
import test_oracle_camera_model as pin_cm
import test_oracle_lm as pin_lm
import test_oracle_normal_eq as pin_neq
import test_oracle_pcg as pin_pcg
import test_oracle_power_series as pin_ps

ORACLE_MODULES = (o_cm, o_neq, o_ps, o_direct, o_lm, o_pcg, o_adj)
# the pins' own modules, some of which import oracle functions by name
PIN_MODULES = (pin_adj, pin_cm, pin_lm, pin_neq, pin_pcg, pin_ps)
# every function and class of those modules as imported, to check that each edit is undone
ORIGINALS = {(m.__name__, k): v for m in ORACLE_MODULES + PIN_MODULES for k, v in vars(m).items()
             if inspect.isfunction(v) or inspect.isclass(v)}


def _pin(fn, *args):
    def run():
        fn(*args)
    run.__name__ = fn.__name__ + (repr(args) if args else "")
    return run


def _pin_mp(fn):
    """A pin that takes pytest's monkeypatch fixture: run it with its own MonkeyPatch."""
    def run():
        mp = pytest.MonkeyPatch()
        try:
            fn(mp)
        finally:
            mp.undo()
    run.__name__ = fn.__name__
    return run


# pins by part
GOLDEN = _pin(pin_cm.test_golden_projections)
ROTATION = _pin(pin_cm.test_rotation_preserves_norm_and_inverts)
SMALL_ANGLE = _pin(pin_cm.test_small_angle_branch_is_continuous)
FD_JAC = _pin(pin_cm.test_jacobians_match_central_differences)
JAC_CLOSED = _pin(pin_cm.test_jacobian_entries_closed_form_at_identity)
NOISE = _pin(pin_cm.test_generator_noise_is_the_residual_at_ground_truth)
ROT_EXPM = _pin(pin_cm.test_rotation_matches_the_matrix_exponential)
WEIGHTED = _pin(pin_cm.test_weighted_cost)
DENSE_BLOCKS = _pin(pin_neq.test_blocks_equal_dense_normal_matrix)
DAMPING = _pin(pin_neq.test_damping_modes)
CHOL = _pin(pin_neq.test_block_cholesky_inverse)
SCHUR_ROUTE = _pin(pin_neq.test_schur_route_equals_full_dense_solve, 1e-4, 0)
SCHUR_ROUTE_M1 = _pin(pin_neq.test_schur_route_equals_full_dense_solve, 1e-2, 1)
PCG_DIRECT = _pin(pin_neq.test_pcg_matches_dense_cholesky)
MODEL_DEC = _pin(pin_neq.test_model_decrease_closed_form)
REDUCED_PCG = _pin(pin_neq.test_solve_reduced_takes_pcg_above_the_dense_limit)
TRUNC2 = _pin(pin_ps.test_truncation_error_identity, 2)
STOP_INDEX = _pin(pin_ps.test_stop_index_matches_dense_partial_sums)
STOP_SCRIPTED = _pin(pin_ps.test_stop_rule_scripted_sequences)
LAMBDA_RULE = _pin(pin_lm.test_lambda_update_rule)
LM_FLOOR = _pin(pin_lm.test_lm_decreases_cost_and_reaches_noise_floor, "direct")
FUNC_TOL = _pin(pin_lm.test_func_tol_stops_early)
LM_REJECT = _pin(pin_lm.test_cost_increasing_trial_steps_are_rejected)
LM_GRAD = _pin(pin_lm.test_gradient_vanishes_at_convergence)
LM_NOT_SPD = _pin_mp(pin_lm.test_failed_factorisations_raise_lambda_like_rejections)
LM_EPS = _pin(pin_lm.test_power_solver_passes_eps_to_the_series)
PCG_EXACT = _pin(pin_pcg.test_pcg_converges_to_the_exact_reduced_solve, "jacobi", 0)
PCG_ORDER0 = _pin(pin_pcg.test_order_zero_power_series_is_the_U_block_preconditioner)
SJ_EXACT = _pin(pin_pcg.test_schur_jacobi_is_exact_for_single_observation_tracks)
ADJ_OBS = _pin(pin_adj.test_obs_gradient_is_the_derivative_of_a_damped_step)
ADJ_W = _pin(pin_adj.test_weight_gradient_at_the_optimum)
ADJ_POWER = _pin(pin_adj.test_power_series_adjoint_converges_to_the_direct_one, 1.0)


@dataclass
class Case:
    id: str
    module: object
    name: str      # function or class in `module`
    old: str       # text that occurs exactly once in its source
    new: str
    pins: tuple


CASES = [
    # camera model (Sec. 4, BAL convention)
    Case("projection_k2_dropped", o_cm, "project",
         "rad = 1.0 + cam[7] * n2 + cam[8] * n2 * n2", "rad = 1.0 + cam[7] * n2", (GOLDEN, JAC_CLOSED)),
    Case("projection_x_sign", o_cm, "project", "px = -P[0] / P[2]", "px = P[0] / P[2]", (GOLDEN,)),
    Case("projection_divides_by_wrong_axis", o_cm, "project", "py = -P[1] / P[2]", "py = -P[1] / P[0]", (GOLDEN,)),
    Case("projection_translation_index", o_cm, "project", "cam[3 + i]", "cam[4 + i]", (GOLDEN,)),
    Case("rotation_transposed", o_cm, "rotate", "kxX[i] * s", "(-kxX[i]) * s", (ROTATION, GOLDEN)),
    Case("rotation_one_minus_cos_dropped", o_cm, "rotate",
         " + k[i] * kdX * (1.0 - c)", "", (ROTATION, GOLDEN)),
    Case("rotation_small_angle_term_dropped", o_cm, "rotate",
         "first = [X[i] + wxX[i] for i in range(3)]", "first = [X[i] for i in range(3)]",
         (SMALL_ANGLE, JAC_CLOSED)),
    Case("small_angle_threshold_too_large", o_cm, "rotate",
         "small = _value(th2) < THETA2_SMALL", "small = _value(th2) < 1e-6", (ROT_EXPM,)),
    Case("cross_product_index", o_cm, "_cross", "a[2] * b[0] - a[0] * b[2]", "a[2] * b[0] - a[0] * b[1]",
         (ROTATION, GOLDEN)),
    Case("dual_cos_derivative_sign", o_cm, "_cos", "-x.d * np.sin(x.v)", "x.d * np.sin(x.v)", (FD_JAC,)),
    Case("dual_sin_derivative", o_cm, "_sin", "x.d * np.cos(x.v)", "x.d * np.sin(x.v)", (FD_JAC,)),
    Case("dual_sqrt_derivative_half_dropped", o_cm, "_sqrt", "(0.5 / s)", "(1.0 / s)", (FD_JAC,)),
    Case("dual_select_derivative_from_other_branch", o_cm, "_where",
         "np.where(mask[..., None], ad, bd)", "np.where(mask[..., None], bd, ad)", (FD_JAC,)),
    Case("dual_product_rule_term_dropped", o_cm, "Dual",
         "self.d * ov[..., None] + od * self.v[..., None]", "self.d * ov[..., None]", (FD_JAC,)),
    Case("dual_quotient_rule_sign", o_cm, "Dual",
         "(self.d - od * q[..., None]) / ov[..., None]", "(self.d + od * q[..., None]) / ov[..., None]",
         (FD_JAC, JAC_CLOSED)),
    Case("jacobian_rows_swapped", o_cm, "linearize",
         "J = np.stack([pi[0].d, pi[1].d], axis=1)", "J = np.stack([pi[1].d, pi[0].d], axis=1)",
         (FD_JAC, JAC_CLOSED)),
    Case("landmark_jacobian_wrong_columns", o_cm, "linearize", "J[:, :, 9:12]", "J[:, :, 6:9]",
         (FD_JAC, JAC_CLOSED)),
    Case("residual_sign", o_cm, "residuals",
         "pi[0] - obs[:, 0], pi[1] - obs[:, 1]", "obs[:, 0] - pi[0], obs[:, 1] - pi[1]", (NOISE, FD_JAC)),
    Case("weight_not_square_rooted_in_r", o_cm, "residuals",
         "r = r * np.sqrt(weights)[:, None]", "r = r * weights[:, None]", (WEIGHTED,)),
    Case("weight_not_square_rooted_in_J", o_cm, "linearize", "sw = np.sqrt(weights)", "sw = weights",
         (WEIGHTED,)),
    Case("weight_on_J_only", o_cm, "linearize", "        r = r * sw[:, None]\n", "", (WEIGHTED, ADJ_OBS)),
    Case("cost_half_dropped", o_cm, "cost", "0.5 * float(", "1.0 * float(", (WEIGHTED,)),
    # normal equation, damping, inverses (Sec. 4.1 eq. normal)
    Case("landmark_column_order", o_neq, "assemble_jacobians",
         "np.arange(3)[None, None, :]", "np.arange(3)[::-1][None, None, :]", (DENSE_BLOCKS,)),
    Case("camera_row_order", o_neq, "assemble_jacobians",
         "rows_p = (2 * o[:, None, None] + np.arange(2)[None, :, None])",
         "rows_p = (2 * o[:, None, None] + np.arange(2)[::-1][None, :, None])", (DENSE_BLOCKS, SCHUR_ROUTE)),
    Case("b_p_sign", o_neq, "NormalEquation", "self.b_p = self.Jps.T @ rv", "self.b_p = -(self.Jps.T @ rv)",
         (DENSE_BLOCKS, SCHUR_ROUTE)),
    Case("b_l_sign", o_neq, "NormalEquation", "self.b_l = self.Jls.T @ rv", "self.b_l = -(self.Jls.T @ rv)",
         (DENSE_BLOCKS, SCHUR_ROUTE)),
    Case("damping_clamp_dropped", o_neq, "damp",
         "diag = np.clip(blocks[:, idx, idx], DAMP_MIN, DAMP_MAX)", "diag = blocks[:, idx, idx]", (DAMPING,)),
    Case("damping_lambda_dropped", o_neq, "damp", "out[:, idx, idx] += lam * diag", "out[:, idx, idx] += diag",
         (DAMPING, SCHUR_ROUTE)),
    Case("damping_mode_ignored", o_neq, "damp", "if damping_mode == 0:", "if True:", (DAMPING, SCHUR_ROUTE_M1)),
    Case("landmark_blocks_undamped", o_neq, "NormalEquation",
         "damp(self.V, lam, damping_mode)", "damp(self.V, 0.0, damping_mode)", (SCHUR_ROUTE,)),
    Case("cholesky_inverse_factor_order", o_neq, "chol_inverse",
         '"nji,njk->nik"', '"nij,nkj->nik"', (CHOL,)),
    Case("cholesky_inverse_transpose_dropped", o_neq, "chol_inverse",
         '"nji,njk->nik"', '"nij,njk->nik"', (CHOL, TRUNC2)),
    # Schur complement and back-substitution (Sec. 4.2 eqs. Sx, Schur, back_substitution)
    Case("schur_rhs_sign", o_neq, "schur_rhs", "ne.b_p - ne.W @", "ne.b_p + ne.W @", (SCHUR_ROUTE,)),
    Case("schur_complement_sign", o_neq, "explicit_schur", "S = _bd_fast(Ulam) - WVW", "S = _bd_fast(Ulam) + WVW",
         (SCHUR_ROUTE,)),
    Case("back_substitution_printed_sign", o_neq, "back_substitute",
         "ne.b_l + ne.W.T @ dx_p", "-ne.b_l + ne.W.T @ dx_p", (SCHUR_ROUTE,)),
    Case("model_decrease_landmark_sign", o_neq, "model_decrease",
         "rv + ne.Jps @ dx_p + ne.Jls @ dx_l", "rv + ne.Jps @ dx_p - ne.Jls @ dx_l", (MODEL_DEC,)),
    Case("model_decrease_reversed", o_neq, "model_decrease",
         "0.5 * float(rv @ rv) - 0.5 * float(rn @ rn)", "0.5 * float(rn @ rn) - 0.5 * float(rv @ rv)",
         (MODEL_DEC, LM_FLOOR)),
    # power series and stop rule (Sec. 4.3 eqs. inverse, S_approx, x_approx, qcriterion)
    Case("series_x0_sign", o_ps, "power_series_solve",
         "t = -apply_blocks(Uinv, b_tilde)", "t = apply_blocks(Uinv, b_tilde)", (TRUNC2,)),
    Case("series_operator_without_V_inverse", o_ps, "apply_P",
         "ne.W @ apply_blocks(Vinv, ne.W.T @ t)", "ne.W @ (ne.W.T @ t)", (TRUNC2, STOP_INDEX)),
    Case("series_operator_without_U_inverse", o_ps, "apply_P",
         "return apply_blocks(Uinv, ne.W @", "return (ne.W @", (TRUNC2, STOP_INDEX)),
    Case("series_one_term_short", o_ps, "power_series_solve",
         "for i in range(1, m_max + 1):", "for i in range(1, m_max):", (TRUNC2,)),
    Case("series_P_applied_to_the_sum", o_ps, "power_series_solve",
         "t = apply_P(ne, Uinv, Vinv, t)", "t = apply_P(ne, Uinv, Vinv, x)", (TRUNC2, STOP_INDEX)),
    Case("series_stop_factor_i", o_ps, "power_series_solve",
         "stop_value = (i + 1) * tn / xn", "stop_value = i * tn / xn", (STOP_INDEX,)),
    Case("stop_test_factor_i", o_ps, "stop_test",
         "(i + 1) * t_norm / x_norm < eps", "i * t_norm / x_norm < eps", (STOP_SCRIPTED,)),
    Case("stop_test_non_strict", o_ps, "stop_test",
         "(i + 1) * t_norm / x_norm < eps", "(i + 1) * t_norm / x_norm <= eps", (STOP_SCRIPTED,)),
    Case("stop_rule_starts_at_zero", o_ps, "run_stop_rule",
         "for i in range(1, m_max + 1):", "for i in range(0, m_max + 1):", (STOP_SCRIPTED,)),
    # exact solves (Prop. 2 limit) and PCG
    Case("dense_solve_sign", o_direct, "solve_dense", "return -sla.cho_solve(", "return sla.cho_solve(",
         (SCHUR_ROUTE, PCG_EXACT)),
    Case("pcg_updates_y_along_z", o_direct, "pcg", "y += alpha * p", "y += alpha * z", (PCG_DIRECT,)),
    Case("reduced_pcg_rhs_sign", o_direct, "solve_reduced",
         "pcg(S, -b_tilde, Minv", "pcg(S, b_tilde, Minv", (REDUCED_PCG,)),
    Case("matrix_free_schur_sign", o_pcg, "schur_apply",
         "apply_blocks(Ulam, t) - ne.W @", "apply_blocks(Ulam, t) + ne.W @", (PCG_EXACT,)),
    Case("pcg_y_along_z", o_pcg, "pcg", "y = y + alpha * p", "y = y + alpha * z", (PCG_EXACT,)),
    Case("matrix_free_pcg_rz_not_carried", o_pcg, "pcg", "        rz = rz_new\n", "", (PCG_EXACT,)),
    Case("schur_jacobi_from_U_blocks", o_pcg, "schur_jacobi_blocks",
         "S = explicit_schur(ne, Ulam, Vinv, dense=False)\n    return block_diagonal(S, ne.n_cams, 9)",
         "return Ulam.copy()", (SJ_EXACT,)),
    Case("pcg_solve_rhs_sign", o_pcg, "pcg_solve", "t), -bt, apply_Minv", "t), bt, apply_Minv", (PCG_EXACT,)),
    Case("pcg_solve_back_substitution_sign", o_pcg, "pcg_solve",
         "back_substitute(ne, Vi, y)", "back_substitute(ne, Vi, -y)", (PCG_EXACT,)),
    Case("power_preconditioner_first_term_without_U_inverse", o_pcg, "power_series_preconditioner",
         "t = apply_blocks(Uinv, r)", "t = r.copy()", (PCG_ORDER0,)),
    Case("power_preconditioner_without_U_inverse_term", o_pcg, "power_series_preconditioner",
         "        z = t.copy()\n", "        z = 0 * t\n", (PCG_ORDER0,)),
    Case("power_preconditioner_one_term_short", o_pcg, "power_series_preconditioner",
         "for _ in range(m):", "for _ in range(m - 1):", (PCG_ORDER0,)),
    # LM loop (Sec. 5.1)
    Case("lambda_update_square", o_lm, "lambda_update",
         "(2.0 * rho - 1.0) ** 3", "(2.0 * rho - 1.0) ** 2", (LAMBDA_RULE,)),
    Case("lambda_update_nu_not_doubled", o_lm, "lambda_update", "nu = 2.0 * nu", "nu = nu", (LAMBDA_RULE,)),
    Case("lambda_update_reject_by_two", o_lm, "lambda_update", "        lam = lam * nu\n", "        lam = lam * 2.0\n",
         (LAMBDA_RULE,)),
    Case("lm_accepts_cost_increase", o_lm, "lm_solve",
         "actual > 0.0 and pred > 0.0", "pred > 0.0", (LM_REJECT,)),
    Case("lm_not_spd_handled_as_accept", o_lm, "lm_solve",
         "lam, nu = lambda_update(lam, nu, False, 0.0)", "lam, nu = lambda_update(lam, nu, True, 0.0)",
         (LM_NOT_SPD,)),
    Case("lm_series_eps_dropped", o_lm, "solve_step",
         "bt, opts.eps, opts.max_inner)", "bt, 0.0, opts.max_inner)", (LM_EPS,)),
    Case("lm_state_not_moved_on_accept", o_lm, "lm_solve",
         "            cams, lms = cams_new, lms_new\n", "", (LM_FLOOR, LM_GRAD)),
    Case("lm_lambda_update_with_inverted_accept", o_lm, "lm_solve",
         "lam, nu = lambda_update(lam, nu, accepted, rho)", "lam, nu = lambda_update(lam, nu, not accepted, rho)",
         (LM_GRAD,)),
    Case("lm_keeps_stale_linearisation", o_lm, "lm_solve",
         "            ne = None\n            if (F_old", "            if (F_old", (LM_GRAD,)),
    Case("lm_step_subtracted", o_lm, "lm_solve",
         "cams_new = cams + dx_p.reshape(nc, 9)", "cams_new = cams - dx_p.reshape(nc, 9)", (LM_FLOOR,)),
    Case("lm_func_tol_inverted", o_lm, "lm_solve",
         "(F_old - F_new) / F_old < opts.func_tol", "(F_old - F_new) / F_old > opts.func_tol", (FUNC_TOL,)),
    # implicit-differentiation adjoint
    Case("adjoint_rhs_sign", o_adj, "adjoint_solve", "rhs = g_p - ne.W @", "rhs = g_p + ne.W @", (ADJ_OBS,)),
    Case("adjoint_landmark_back_substitution_sign", o_adj, "adjoint_solve",
         "g_l - ne.W.T @ a_p", "g_l + ne.W.T @ a_p", (ADJ_OBS,)),
    Case("adjoint_weights_not_passed", o_adj, "gradients",
         "observation_gradients(r, Jp, Jl, p.weights,", "observation_gradients(r, Jp, Jl, None,", (ADJ_OBS,)),
    Case("adjoint_series_rhs_sign", o_adj, "adjoint_solve",
         "power_series_solve(ne, Ui, Vi, -rhs,", "power_series_solve(ne, Ui, Vi, rhs,", (ADJ_POWER,)),
    Case("adjoint_obs_gradient_sign", o_adj, "observation_gradients",
         "d_obs = np.sqrt(w)[:, None] * u", "d_obs = -np.sqrt(w)[:, None] * u", (ADJ_OBS,)),
    Case("adjoint_damping_mode_flipped", o_adj, "adjoint_solve",
         "ne.damped(lam, damping_mode)", "ne.damped(lam, 1 - damping_mode)", (ADJ_OBS, ADJ_W)),
    Case("adjoint_landmark_part_dropped", o_adj, "observation_gradients",
         ' + np.einsum("oij,oj->oi", Jl, al)', "", (ADJ_OBS, ADJ_W)),
    Case("adjoint_obs_weight_dropped", o_adj, "observation_gradients",
         "d_obs = np.sqrt(w)[:, None] * u", "d_obs = u", (ADJ_OBS,)),
    Case("adjoint_weight_gradient_sign", o_adj, "observation_gradients",
         "d_w = -np.sum(r * u, axis=1) / w", "d_w = np.sum(r * u, axis=1) / w", (ADJ_W,)),
]


def _plant(case, monkeypatch):
    """Compile `case.name` with the one-line edit and install it wherever the oracle refers to
    the original object."""
    orig = getattr(case.module, case.name)
    src = textwrap.dedent(inspect.getsource(orig))
    n = src.count(case.old)
    assert n == 1, f"{case.module.__name__}.{case.name}: edit site {case.old!r} occurs {n} times"
    code = compile(src.replace(case.old, case.new), f"<planted {case.id}>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    # Define the edited version in the module's own namespace, so that it sees the module's
    # globals as they are at call time (including any a pin patches), then put the original
    # back and install the edit through monkeypatch, which undoes it after the test.
    exec(code, vars(case.module))
    mutant = getattr(case.module, case.name)
    setattr(case.module, case.name, orig)
    for mod in ORACLE_MODULES + PIN_MODULES:
        if getattr(mod, case.name, None) is orig:
            monkeypatch.setattr(mod, case.name, mutant)


@pytest.mark.parametrize("case", CASES, ids=[c.id for c in CASES])
def test_planted_mistake_fails_a_pin(case, monkeypatch):
    _plant(case, monkeypatch)
    missed = []
    for pin in case.pins:
        try:
            with np.errstate(all="ignore"):  # some edits overflow on purpose
                pin()
        except AssertionError:
            continue
        missed.append(pin.__name__)
    assert not missed, f"planted mistake {case.id} passed {missed}"


def test_pins_pass_without_a_planted_mistake():
    pins = {p.__name__: p for c in CASES for p in c.pins}
    for name, pin in sorted(pins.items()):
        pin()


def test_every_edit_was_undone():
    """Runs after the cases above: each module again holds the objects it was imported with."""
    mods = {m.__name__: m for m in ORACLE_MODULES + PIN_MODULES}
    changed = [key for key, v in ORIGINALS.items() if vars(mods[key[0]]).get(key[1]) is not v]
    assert not changed, changed
