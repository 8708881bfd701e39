"""GPU implicit-differentiation adjoint against the FP64 oracle (oracle/adjoint.py): the same
series (equal lambda, eps, m) within 1e-10 relative in FP64 and 1e-4 in FP32-bulk, the exact
reduced solve within 1e-8 once the series has converged, device and host buffers alike, the
torch.autograd.Function, a finite-difference check through the re-solved regularised
minimiser, and the weighted 200-camera / 20,000-landmark workload."""
import numpy as np
import pytest

import bal_synth
from gpu_helpers import rel
from oracle import adjoint as oad
from oracle import camera_model as cm
from oracle import normal_eq as neq

pytestmark = pytest.mark.gpu


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
def solved(poba):
    """A weighted problem after 12 GPU LM iterations (the state the adjoint is taken at)."""
    p = bal_synth.make_problem(30, 800, track=("uniform", 2, 6), weighted=True, seed=301)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights,
                       options=poba.ba_default_options(max_lm=12))
    poba.ba_lm_solve(h, max_lm=12)
    cams, lms = poba.ba_get_params(h)
    return p, cams, lms


def grads(p, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(p.n_cams, 9)), rng.normal(size=(p.n_lms, 3))


def handle_at(poba, p, cams, lms, precision=0, **opt):
    h = poba.ba_create(cams, lms, p.obs, p.cam_idx, p.lm_idx, p.weights, precision=precision,
                       options=poba.ba_default_options(**opt))
    return h


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("lam,m", [(1e-2, 30), (1.0, 5)])
def test_adjoint_matches_oracle_series(poba, solved, precision, tol, lam, m):
    p, cams, lms = solved
    g_c, g_l = grads(p, 1)
    h = handle_at(poba, p, cams, lms, precision, eps=0.0, max_inner=m)
    d_obs, d_w, info = poba.ba_adjoint(h, lam, g_c, g_l)
    assert info["inner_iters"] == m
    o_obs, o_w, a_p, a_l, om = oad.gradients(p, cams, lms, g_c, g_l, lam, solver="power", eps=0.0,
                                             m_max=m)
    assert om == m
    assert rel(d_obs, o_obs) < tol, rel(d_obs, o_obs)
    assert rel(d_w, o_w) < tol, rel(d_w, o_w)
    # the adjoint vector is left in the step buffers
    a_pg, a_lg = poba.ba_get_step(h)
    assert rel(a_pg, a_p) < tol and rel(a_lg, a_l) < tol


def test_adjoint_converged_series_matches_exact_solve(poba, solved):
    p, cams, lms = solved
    g_c, g_l = grads(p, 2)
    lam = 0.1
    h = handle_at(poba, p, cams, lms, eps=1e-14, max_inner=600)
    d_obs, d_w, info = poba.ba_adjoint(h, lam, g_c, g_l)
    o_obs, o_w, _, _, _ = oad.gradients(p, cams, lms, g_c, g_l, lam, solver="direct")
    assert rel(d_obs, o_obs) < 1e-8 and rel(d_w, o_w) < 1e-8, (rel(d_obs, o_obs), info)


def test_adjoint_device_buffers_and_stop_rule(poba, solved):
    import torch
    p, cams, lms = solved
    g_c, g_l = grads(p, 3)
    h = handle_at(poba, p, cams, lms, eps=0.01, max_inner=20)
    a_obs, a_w, ia = poba.ba_adjoint(h, 1.0, g_c, g_l)
    dev = torch.device("cuda")
    b_obs, b_w, ib = poba.ba_adjoint(h, 1.0, torch.as_tensor(g_c, device=dev),
                                     torch.as_tensor(g_l, device=dev))
    assert b_obs.is_cuda and b_w.is_cuda
    assert np.array_equal(a_obs, b_obs.cpu().numpy()) and np.array_equal(a_w, b_w.cpu().numpy())
    o = oad.gradients(p, cams, lms, g_c, g_l, 1.0, solver="power", eps=0.01, m_max=20)
    assert ia["inner_iters"] == ib["inner_iters"] == o[4] < 20
    assert rel(a_obs, o[0]) < 1e-10
    # without weights the weight gradient is optional
    _, none_w, _ = poba.ba_adjoint(h, 1.0, g_c, g_l, want_weights=False)
    assert none_w is None


def test_autograd_function(poba):
    """bundle_adjust: forward runs LM to convergence, backward the adjoint at the given lambda;
    the gradients equal the oracle's at the converged state."""
    import torch
    from paper_2204_12834_gb300.autograd import bundle_adjust
    p = bal_synth.make_problem(20, 500, track=("uniform", 3, 5), weighted=True, seed=303)
    dev = torch.device("cuda")
    obs = torch.tensor(p.obs, device=dev, requires_grad=True)
    w = torch.tensor(p.weights, device=dev, requires_grad=True)
    lam = 0.05
    adj = poba.ba_default_options(eps=1e-14, max_inner=800)
    cams, lms = bundle_adjust(obs, torch.tensor(p.cams0, device=dev), torch.tensor(p.lms0, device=dev),
                              torch.tensor(p.cam_idx, device=dev), torch.tensor(p.lm_idx, device=dev),
                              weights=w, options=poba.ba_default_options(max_lm=30),
                              adjoint_lambda=lam, adjoint_options=adj)
    g_c, g_l = grads(p, 4)
    loss = (cams * torch.tensor(g_c, device=dev)).sum() + (lms * torch.tensor(g_l, device=dev)).sum()
    loss.backward()
    c, l = cams.detach().cpu().numpy(), lms.detach().cpu().numpy()
    o_obs, o_w, _, _, _ = oad.gradients(p, c, l, g_c, g_l, lam, solver="direct")
    assert rel(obs.grad.cpu().numpy(), o_obs) < 1e-8
    assert rel(w.grad.cpu().numpy(), o_w) < 1e-8


def test_finite_difference_through_regularised_minimiser(poba):
    """With noise-free observations (r = 0 at the ground truth) the GPU adjoint gradient equals
    the finite difference of argmin F + lam/2 ||D (x - x_gt)||^2, the minimiser with the gauge
    fixed by a prior at the same lambda."""
    from test_oracle_adjoint import regularised_minimiser
    p = bal_synth.make_problem(5, 40, track=("uniform", 3, 5), pixel_noise=0.0, seed=305)
    cams, lms = p.cams_gt, p.lms_gt
    lam = 1e-2
    r, Jp, Jl = cm.linearize(cams, lms, p.obs, p.cam_idx, p.lm_idx)
    ne = neq.NormalEquation(r, Jp, Jl, p.cam_idx, p.lm_idx, p.n_cams, p.n_lms)
    idx9, idx3 = np.arange(9), np.arange(3)
    D2 = np.concatenate([np.clip(ne.U[:, idx9, idx9], neq.DAMP_MIN, neq.DAMP_MAX).ravel(),
                         np.clip(ne.V[:, idx3, idx3], neq.DAMP_MIN, neq.DAMP_MAX).ravel()])
    g_c, g_l = grads(p, 5)
    g = np.concatenate([g_c.ravel(), g_l.ravel()])
    h = handle_at(poba, p, cams, lms, eps=1e-15, max_inner=2000)
    d_obs, _, _ = poba.ba_adjoint(h, lam, g_c, g_l)
    rng = np.random.default_rng(6)
    step = 1e-4
    for o in rng.choice(p.n_obs, 6, replace=False):
        for i in range(2):
            ob = p.obs.copy()
            ob[o, i] += step
            fp = g @ regularised_minimiser(p, ob, cams, lms, lam, D2)
            ob[o, i] -= 2 * step
            fm = g @ regularised_minimiser(p, ob, cams, lms, lam, D2)
            fd = (fp - fm) / (2 * step)
            assert abs(fd - d_obs[o, i]) <= 1e-5 * max(abs(fd), 1e-2 * np.abs(d_obs).max())


def test_adjoint_weighted_200c_20000l(poba):
    """The differentiable workload: 200 cameras, 20,000 landmarks (about 80,000 observations),
    weights U(0.5, 1.5), FP64.  LM to convergence, then the adjoint at lambda = 1e-2 with 40
    terms, against the oracle's series gradient on every observation."""
    p = bal_synth.preset("weighted_200c_20000l")
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    poba.ba_lm_solve(h)
    cams, lms = poba.ba_get_params(h)
    poba.ba_set_options(h, poba.ba_default_options(eps=0.0, max_inner=40))
    g_c, g_l = grads(p, 7)
    d_obs, d_w, info = poba.ba_adjoint(h, 1e-2, g_c, g_l)
    o_obs, o_w, _, _, m = oad.gradients(p, cams, lms, g_c, g_l, 1e-2, solver="power", eps=0.0,
                                        m_max=40)
    assert info["inner_iters"] == m == 40
    assert rel(d_obs, o_obs) < 1e-10 and rel(d_w, o_w) < 1e-10


def test_autograd_backward_restores_options_and_flags_truncation(poba, monkeypatch):
    """The backward applies adjoint_options to its own solve only: the handle gets the forward's
    options back afterwards.  A series cut at its term cap (2 terms, eps 1e-14) raises a
    RuntimeWarning and leaves its state in BundleAdjustment.last_adjoint_info."""
    import torch
    from paper_2204_12834_gb300 import autograd as ag
    p = bal_synth.make_problem(12, 300, track=("uniform", 3, 5), weighted=True, seed=306)
    dev = torch.device("cuda")
    obs = torch.tensor(p.obs, device=dev, requires_grad=True)
    fwd = poba.ba_default_options(max_lm=10, eps=0.02)
    adj = poba.ba_default_options(eps=1e-14, max_inner=2)
    calls = []
    real = ag.ba_set_options
    monkeypatch.setattr(ag, "ba_set_options",
                        lambda h, o: (calls.append((o.eps, o.max_inner, o.max_lm)), real(h, o)))
    cams, lms = ag.bundle_adjust(obs, torch.tensor(p.cams0, device=dev),
                                 torch.tensor(p.lms0, device=dev),
                                 torch.tensor(p.cam_idx, device=dev),
                                 torch.tensor(p.lm_idx, device=dev),
                                 options=fwd, adjoint_lambda=1e-3, adjoint_options=adj)
    with pytest.warns(RuntimeWarning, match="truncated"):
        (cams.sum() + lms.sum()).backward()
    assert calls == [(1e-14, 2, adj.max_lm), (0.02, fwd.max_inner, 10)]
    info = ag.BundleAdjustment.last_adjoint_info
    assert info["inner_iters"] == 2 and not info["stopped"]
    assert torch.isfinite(obs.grad).all()
