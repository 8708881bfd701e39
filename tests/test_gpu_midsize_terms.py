"""Every series term and stop value against the oracle on a mid-size power-law problem.

The 10,000-camera power-law benchmark problem is too large for the oracle to follow term by
term, so this problem reproduces its shape at a tenth of the size: 1,000 cameras, 100,000
landmarks, power-law track lengths on [2, 50] (exponent 2.14), clustered visibility with window
max(2k, 64) -- about 500,000 observations, with many group slots per group and several partial
rows per camera, as on the large problem.  At lambda = 1e-3 and for m = 0 .. 20 (Sec. 4.3, eq.
`x_approx`; eps = 0 so that exactly m terms run) the GPU's x(m) matches the oracle's term
recursion (whole-vector and per-block), and its stop value (m + 1) ||t_m|| / ||x(m)|| (eq.
`qcriterion`) matches the oracle's; then the default rule (eps = 0.01) stops at the oracle's
term.  FP64 and FP32 bulk."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import OracleRef, check_step_blocks, rel
from oracle import normal_eq as neq
from oracle import power_series as ps

pytestmark = pytest.mark.gpu

LAM = 1e-3
M_MAX = 20


@pytest.fixture(scope="module")
def poba():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    m.library()
    return m


@pytest.fixture(scope="module")
def case():
    """The problem and the oracle's x(i), landmark steps and stop values for i = 0 .. 20."""
    p = bal_synth.make_problem(1000, 100000, track=("powerlaw", 2.14, 2, 50),
                               visibility="clustered", window=64, seed=1013)
    ref = OracleRef(p)
    Ul, Vl = ref.ne.damped(LAM, 0)
    Ui, Vi = neq.chol_inverse(Ul), neq.chol_inverse(Vl)
    bt = neq.schur_rhs(ref.ne, Vi)
    t = -neq.apply_blocks(Ui, bt)
    x = t.copy()
    xs, svs = [x.copy()], [np.inf]
    for i in range(1, M_MAX + 1):
        t = ps.apply_P(ref.ne, Ui, Vi, t)
        x = x + t
        xs.append(x.copy())
        svs.append((i + 1) * np.linalg.norm(t) / np.linalg.norm(x))
    xls = [neq.back_substitute(ref.ne, Vi, xi) for xi in xs]
    return p, ref, xs, xls, svs


def test_problem_has_the_large_problems_shape(poba, case):
    """Several group slots per group and several partial rows per camera, as on the large
    power-law problem."""
    p = case[0]
    assert 400_000 < p.n_obs < 600_000
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=1)
    s = poba.ba_get_schedule(h)
    assert s["n_group_slots"] / s["n_groups"] > 20
    assert s["n_group_slots"] / p.n_cams > 3


@pytest.mark.parametrize("precision,tol,sv_tol", [(0, 1e-10, 1e-8), (1, 1e-4, 1e-3)])
def test_every_term_and_stop_value(poba, case, precision, tol, sv_tol):
    p, ref, xs, xls, svs = case
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=precision,
                       options=poba.ba_default_options(eps=0.0, max_inner=0))
    poba.ba_linearize(h)
    for m in range(M_MAX + 1):
        poba.ba_set_options(h, poba.ba_default_options(eps=0.0, max_inner=m))
        info = poba.ba_solve_schur_power(h, LAM)
        assert info["inner_iters"] == m
        dxp, dxl = poba.ba_get_step(h)
        assert rel(dxp, xs[m]) < tol, (m, rel(dxp, xs[m]))
        assert rel(dxl, xls[m]) < tol, (m, rel(dxl, xls[m]))
        check_step_blocks(dxp, dxl, xs[m], xls[m], precision)
        if m == 0:
            assert info["stop_value"] == np.inf
        else:
            assert abs(info["stop_value"] - svs[m]) <= sv_tol * svs[m], (m, info["stop_value"], svs[m])
        assert abs(info["x_norm"] - np.linalg.norm(xs[m])) <= tol * np.linalg.norm(xs[m])


@pytest.mark.parametrize("series_exec", [2, 3, 5, 1])
def test_stop_rule_term_fp64(poba, case, series_exec):
    """eps = 0.01: the rule fires at the oracle's term in every execution form."""
    p, ref, xs, xls, svs = case
    want = next((i for i in range(1, M_MAX + 1) if svs[i] < 0.01), M_MAX)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx,
                       options=poba.ba_default_options(eps=0.01, max_inner=M_MAX,
                                                       series_exec=series_exec))
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_power(h, LAM)
    assert info["inner_iters"] == want
    assert info["stopped"] == (1 if svs[want] < 0.01 else 0)
    dxp, _ = poba.ba_get_step(h)
    assert rel(dxp, xs[want]) < 1e-10
