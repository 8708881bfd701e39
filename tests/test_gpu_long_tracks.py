"""Tracks of more than 256 observations (the long tracks of the BAL problems, Sec. 5 "Dataset")
against the FP64 oracle, which treats every landmark whole.

The library splits such a track into near-equal pieces of at most 256 observations; the pieces
carry copies of the landmark's state and their landmark-side sums are added in piece order.
These tests check that the split is invisible in the results: the blocks V and b_l of Sec. 4.1,
the series x(m) of Sec. 4.3 at fixed m and with the stop rule, the back-substituted landmark
step, LM iterations (Sec. 5.1), PCG on the reduced system and the adjoint gradients -- FP64 at
the usual 1e-10 / 1e-12, FP32 bulk at 1e-4 -- and that every series form agrees bit for bit."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import OracleRef, check_step_blocks, rel
from oracle import lm as olm

pytestmark = pytest.mark.gpu

LONG = (300, 700, 2000, 257, 512)


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
def problem():
    # about 60 observations per camera besides the long tracks, so that the float32 error of the
    # FP32-bulk series at small lambda stays within its bound (a camera seen a handful of times
    # is poorly conditioned, long tracks or not)
    p = bal_synth.make_problem(2100, 30000, track=("long", 2, 6, LONG), weighted=True, seed=1201)
    counts = np.bincount(p.lm_idx)
    assert sorted(counts[counts > 256]) == sorted(k for k in LONG if k > 256)
    return p


@pytest.fixture(scope="module")
def small_long():
    """Two long tracks on 320 cameras: small enough for the oracle's explicit Schur complement
    (a track of k views couples k^2 / 2 camera pairs)."""
    return bal_synth.make_problem(320, 600, track=("long", 2, 6, (300, 270)), weighted=True,
                                  seed=1202)


@pytest.fixture(scope="module")
def ref(problem):
    return OracleRef(problem)


def make(poba, p, precision=0, **opt):
    return poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights,
                          precision=precision, options=poba.ba_default_options(**opt))


def test_blocks_fp64(poba, problem, ref):
    h = make(poba, problem)
    cost = poba.ba_linearize(h)
    U, V, bp, bl = poba.ba_get_blocks(h)
    assert np.abs(U - ref.ne.U).max() / np.abs(ref.ne.U).max() < 1e-12
    assert np.abs(V - ref.ne.V).max() / np.abs(ref.ne.V).max() < 1e-12
    assert rel(bp, ref.ne.b_p) < 1e-12
    assert rel(bl, ref.ne.b_l) < 1e-12
    assert abs(cost - 0.5 * np.sum(ref.r ** 2)) <= 1e-12 * cost
    # the long tracks' own blocks, one by one
    for l in np.nonzero(np.bincount(problem.lm_idx) > 256)[0]:
        assert np.abs(V[l] - ref.ne.V[l]).max() <= 1e-12 * np.abs(ref.ne.V[l]).max()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("lam,m", [(1e-3, 6), (1e-2, 0), (1e-4, 20)])
def test_series_at_fixed_m(poba, problem, ref, precision, tol, lam, m):
    h = make(poba, problem, precision, eps=0.0, max_inner=m)
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_power(h, lam)
    assert info["inner_iters"] == m
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(lam, 0.0, m)
    assert rel(dxp, o["x"]) < tol, rel(dxp, o["x"])
    assert rel(dxl, o["xl"]) < tol, rel(dxl, o["xl"])
    check_step_blocks(dxp, dxl, o["x"], o["xl"], precision)
    if precision == 0:
        long_l = np.nonzero(np.bincount(problem.lm_idx) > 256)[0]
        xl = dxl.reshape(-1, 3)[long_l]
        ox = o["xl"].reshape(-1, 3)[long_l]
        assert np.abs(xl - ox).max() <= 1e-10 * np.abs(ox).max()


def test_stop_rule_fp64(poba, problem, ref):
    o = ref.solve(1.0, 0.01, 20)
    h = make(poba, problem, eps=0.01, max_inner=20)
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_power(h, 1.0)
    assert info["inner_iters"] == o["m"]
    assert abs(info["stop_value"] - o["sv"]) <= 1e-8 * o["sv"]


@pytest.mark.parametrize("precision", [0, 1])
def test_series_forms_agree_bitwise(poba, problem, precision):
    """Per-term launches (0), their graph (1), the persistent kernel (3); forms 4 and 5 fall
    back to 3 on a problem with long tracks; the handle's choice (2)."""
    res = []
    for mode in (0, 1, 2, 3, 4, 5):
        h = make(poba, problem, precision, eps=0.01, max_inner=12, series_exec=mode)
        poba.ba_linearize(h)
        info = poba.ba_solve_schur_power(h, 1e-2)
        res.append((info["inner_iters"], poba.ba_get_step(h)))
    for r in res[1:]:
        assert r[0] == res[0][0]
        assert np.array_equal(r[1][0], res[0][1][0]) and np.array_equal(r[1][1], res[0][1][1])


def test_schedule_rejects_forms_4_and_5(poba, problem):
    h = make(poba, problem, precision=1)
    for form in (4, 5):
        with pytest.raises(poba.PobaError) as e:
            poba.ba_set_schedule(h, series_exec=form, blocks_per_sm=1)
        assert e.value.status_name == "BA_ERR_INVALID_ARG"
    assert poba.ba_autotune(h, trials=1)["exec"] in (1, 3)


def test_lm_iterations_match_oracle(poba, problem):
    """Six LM iterations (eps 1e-10): the same accept / reject decisions and series lengths,
    costs within 1e-6; the state stays consistent across the pieces (get / set round trip)."""
    n = 6
    cams, lms, hist = olm.lm_solve(problem, olm.Options(max_lm=n, eps=1e-10, func_tol=0.0))
    h = make(poba, problem, eps=1e-10, func_tol=0.0)
    steps = [poba.ba_lm_step(h) for _ in range(len(hist))]
    for s, o in zip(steps, hist):
        assert s["accepted"] == o["accepted"]
        assert s["inner"] == o["inner"]
        assert abs(s["cost_after"] - o["cost_after"]) <= 1e-6 * o["cost_after"]
    c, l = poba.ba_get_params(h)
    assert np.abs(l - lms).max() <= 1e-6 * np.abs(lms).max()
    assert np.abs(c - cams).max() <= 1e-6 * np.abs(cams).max()
    poba.ba_set_params(h, c, l)
    c2, l2 = poba.ba_get_params(h)
    assert np.array_equal(c2, c) and np.array_equal(l2, l)
    assert abs(poba.ba_cost(h) - steps[-1]["cost_after" if steps[-1]["accepted"] else "cost_before"]) \
        <= 1e-12 * poba.ba_cost(h)


def test_pcg_matches_direct_solve(poba, small_long):
    """PCG with the Schur-Jacobi preconditioner to 1e-12 against the oracle's direct solve."""
    lam = 1e-3
    problem = small_long
    ref = OracleRef(problem)
    h = make(poba, problem)
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_pcg(h, lam, "jacobi", rtol=1e-12, max_iter=2000)
    assert info["converged"]
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(lam, 0.0, 0)
    from oracle import direct, normal_eq as neq
    Ul, Vl = ref.ne.damped(lam, 0)
    Vi = neq.chol_inverse(Vl)
    x = direct.solve_reduced(ref.ne, Ul, Vi, o["bt"])
    xl = neq.back_substitute(ref.ne, Vi, x)
    assert rel(dxp, x) < 1e-8 and rel(dxl, xl) < 1e-8


def test_adjoint_gradient_matches_oracle(poba, small_long):
    """The implicit-differentiation gradient at lambda = 1e-2 against the oracle's adjoint with
    the same truncated series (eps 1e-14, at most 400 terms)."""
    from oracle import adjoint as oad
    lam = 1e-2
    problem = small_long
    rng = np.random.default_rng(7)
    g_c = rng.normal(size=(problem.n_cams, 9))
    g_l = rng.normal(size=(problem.n_lms, 3))
    h = make(poba, problem, eps=1e-14, max_inner=400)
    d_obs, d_w, info = poba.ba_adjoint(h, lam, g_c, g_l)
    o_obs, o_w, _, _, m = oad.gradients(problem, problem.cams0, problem.lms0, g_c, g_l, lam,
                                        solver="power", eps=1e-14, m_max=400)
    assert info["inner_iters"] == m
    assert rel(d_obs, o_obs) < 1e-8
    assert rel(d_w, o_w) < 1e-8
