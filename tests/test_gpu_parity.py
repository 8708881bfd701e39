"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
problems.  Tolerances: FP64 mode -- series / step relative difference <= 1e-10 at equal
(lambda, m), residuals, Jacobians and blocks <= 1e-12 relative (measured <= 1e-14: FP64 rounding
of the projection and its chain rule, with r = pi - obs cancelling against pixel-sized
observations); FP32-bulk mode -- series relative difference <= 1e-4; LM final cost within 1e-6
relative."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import FP32_BLOCK_TOL, FP64_BLOCK_TOL, OracleRef, block_rel, rel

pytestmark = pytest.mark.gpu

FP64_SERIES_TOL = 1e-10
FP32_SERIES_TOL = 1e-4
LIN_TOL = 1e-12

# series group sizes (observations per group; ba_set_schedule): the automatic size (one group
# per block, on these problems a single chunk), groups of a few chunks, and one group per
# problem (every chunk of the problem accumulates into one set of group slots)
GROUP_SIZES = [0, 700, 1 << 30]


@pytest.fixture(scope="module")
def poba():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    m.library()
    return m


def make(poba, p, precision=0, group_obs=0, **opt):
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights,
                       precision=precision, options=poba.ba_default_options(**opt))
    if group_obs:
        poba.ba_set_schedule(h, group_obs=group_obs)
    return h


def check_blocks(dxp, dxl, o, tol):
    assert block_rel(dxp, o["x"], 9) < tol
    assert block_rel(dxl, o["xl"], 3) < tol


PROBLEMS = {
    "uniform_16c_1000l": lambda: bal_synth.preset("uniform_16c_1000l"),
    "clustered_60c_3000l": lambda: bal_synth.make_problem(60, 3000, track=("uniform", 3, 4),
                                                          visibility="clustered", seed=77),
    "uniform_200c_2000l_weighted": lambda: bal_synth.make_problem(200, 2000, track=("uniform", 2, 6),
                                                                  weighted=True, seed=78),
    "powerlaw_80c_2000l": lambda: bal_synth.make_problem(80, 2000, track=("powerlaw", 2.14, 2, 50),
                                                         visibility="clustered", window=64, seed=79),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    return request.param, p, OracleRef(p)


def test_linearization_fp64(poba, case):
    name, p, ref = case
    h = make(poba, p)
    cost = poba.ba_linearize(h)
    r, Jp, Jl = poba.ba_get_linearization(h)
    assert rel(r, ref.r) < LIN_TOL
    assert np.abs(Jp - ref.Jp).max() / np.abs(ref.Jp).max() < LIN_TOL
    assert np.abs(Jl - ref.Jl).max() / np.abs(ref.Jl).max() < LIN_TOL
    assert abs(cost - 0.5 * np.sum(ref.r ** 2)) / cost < 1e-12


def test_blocks_fp64(poba, case):
    name, p, ref = case
    h = make(poba, p)
    poba.ba_linearize(h)
    U, V, bp, bl = poba.ba_get_blocks(h)
    assert np.abs(U - ref.ne.U).max() / np.abs(ref.ne.U).max() < LIN_TOL
    assert np.abs(V - ref.ne.V).max() / np.abs(ref.ne.V).max() < LIN_TOL
    assert rel(bp, ref.ne.b_p) < LIN_TOL
    assert rel(bl, ref.ne.b_l) < LIN_TOL


@pytest.mark.parametrize("group_obs", GROUP_SIZES)
@pytest.mark.parametrize("lam,m", [(1e-4, 20), (1e-2, 5), (1.0, 0), (1e-3, 1)])
def test_series_fp64_at_fixed_m(poba, case, lam, m, group_obs):
    name, p, ref = case
    h = make(poba, p, eps=0.0, max_inner=m, group_obs=group_obs)
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_power(h, lam)
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(lam, 0.0, m)
    assert info["inner_iters"] == o["m"] == m
    assert rel(dxp, o["x"]) < FP64_SERIES_TOL
    assert rel(dxl, o["xl"]) < FP64_SERIES_TOL
    check_blocks(dxp, dxl, o, FP64_BLOCK_TOL)
    # the normal-equation residual of the GPU step equals the oracle's
    rg, ro = ref.schur_residual(lam, dxp.ravel()), ref.schur_residual(lam, o["x"])
    assert abs(rg - ro) <= 1e-8 * max(ro, 1e-300) + 1e-14


@pytest.mark.parametrize("group_obs", GROUP_SIZES)
def test_series_stop_rule_fp64(poba, case, group_obs):
    name, p, ref = case
    lam = 1.0  # small spectral radius: the rule fires well before m_max
    o = ref.solve(lam, 0.01, 20)
    h = make(poba, p, eps=0.01, max_inner=20, group_obs=group_obs)
    poba.ba_linearize(h)
    info = poba.ba_solve_schur_power(h, lam)
    assert info["inner_iters"] == o["m"]
    assert info["stopped"] == (1 if o["m"] < 20 or o["sv"] < 0.01 else 0)
    assert abs(info["stop_value"] - o["sv"]) <= 1e-8 * o["sv"]
    dxp, _ = poba.ba_get_step(h)
    assert rel(dxp, o["x"]) < FP64_SERIES_TOL


@pytest.mark.parametrize("group_obs", GROUP_SIZES)
@pytest.mark.parametrize("lam,m", [(1e-4, 20), (1e-2, 5)])
def test_series_fp32_bulk(poba, case, lam, m, group_obs):
    name, p, ref = case
    h = make(poba, p, precision=1, eps=0.0, max_inner=m, group_obs=group_obs)
    poba.ba_linearize(h)
    poba.ba_solve_schur_power(h, lam)
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(lam, 0.0, m)
    assert rel(dxp, o["x"]) < FP32_SERIES_TOL
    assert rel(dxl, o["xl"]) < FP32_SERIES_TOL
    check_blocks(dxp, dxl, o, FP32_BLOCK_TOL)


def test_damping_identity_mode(poba, case):
    name, p, ref = case
    h = make(poba, p, eps=0.0, max_inner=6, damping_mode=1)
    poba.ba_linearize(h)
    poba.ba_solve_schur_power(h, 10.0)
    dxp, dxl = poba.ba_get_step(h)
    o = ref.solve(10.0, 0.0, 6, damping_mode=1)
    assert rel(dxp, o["x"]) < FP64_SERIES_TOL
    assert rel(dxl, o["xl"]) < FP64_SERIES_TOL


def test_cost_fp64(poba, case):
    from oracle import camera_model as cm
    name, p, ref = case
    for prec in (0, 1):
        h = make(poba, p, precision=prec)
        c = poba.ba_cost(h)
        co = cm.cost(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
        assert abs(c - co) / co < 1e-12


def test_solve_is_deterministic(poba, case):
    name, p, ref = case
    out = []
    for _ in range(2):
        h = make(poba, p, eps=0.0, max_inner=7)
        poba.ba_linearize(h)
        poba.ba_solve_schur_power(h, 1e-3)
        out.append(poba.ba_get_step(h))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("group_obs", GROUP_SIZES)
@pytest.mark.parametrize("precision", [0, 1])
def test_series_exec_modes_agree_bitwise(poba, case, precision, group_obs):
    """Per-kernel launches, the captured graph, the persistent kernel (series_exec 3), the
    persistent kernel with staged chunks (4; FP64 runs it as 3), the dataflow persistent kernel
    (5) and the handle's own choice give the same step for one series schedule."""
    name, p, ref = case
    res = []
    for mode in (0, 1, 2, 3, 4, 5):
        h = make(poba, p, precision=precision, eps=0.01, max_inner=12, series_exec=mode,
                 group_obs=group_obs)
        poba.ba_linearize(h)
        info = poba.ba_solve_schur_power(h, 1e-2)
        res.append((info["inner_iters"], poba.ba_get_step(h)))
    for r in res[1:]:
        assert r[0] == res[0][0]
        assert np.array_equal(r[1][0], res[0][1][0]) and np.array_equal(r[1][1], res[0][1][1])


def test_autotune_keeps_results(poba, case):
    """ba_autotune times the series schedules and keeps one; the options are unchanged, the
    schedule it reports is in force, and the tuned handle's step equals the graph-replay step of
    a handle given the same group size, bit for bit, and the oracle's to 1e-10 (FP64)."""
    name, p, ref = case
    for precision in (0, 1):
        h = make(poba, p, precision=precision, eps=0.01, max_inner=12)
        poba.ba_linearize(h)
        choice = poba.ba_autotune(h, trials=2)
        sched = poba.ba_get_schedule(h)
        assert choice["exec"] in (1, 3, 4, 5) and (choice["exec"] != 4 or precision == 1)
        assert sched["series_exec"] == choice["exec"] and sched["group_obs"] >= 256
        assert sched["n_groups"] >= 1 and sched["n_group_slots"] >= 1
        assert poba.ba_default_options().eps == 0.01
        info = poba.ba_solve_schur_power(h, 1e-2)
        g = make(poba, p, precision=precision, eps=0.01, max_inner=12, series_exec=1,
                 group_obs=sched["group_obs"])
        poba.ba_linearize(g)
        info_g = poba.ba_solve_schur_power(g, 1e-2)
        assert info["inner_iters"] == info_g["inner_iters"]
        a, b = poba.ba_get_step(h), poba.ba_get_step(g)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        if precision == 0:
            o = ref.solve(1e-2, 0.01, 12)
            assert rel(a[0], o["x"]) < FP64_SERIES_TOL
