"""The allocation-free cost entry point (ba_cost_noalloc) against the oracle's float64 cost.

ba_cost_noalloc serves callers that must not let a library allocate device memory (cudaMalloc
and cudaFree synchronise the device; some processes hand all device memory to one allocator).
It keeps its scratch in one fixed device array shared by all calls.  This test checks:
  * two calls in a row on different problems, each against the oracle's F (Sec. 4) and against
    the handle-based ba_cost, to 1e-12 relative, then the first problem again (no state leaks);
  * the documented edge cases: n_obs = 0 gives 0.0, an out-of-range camera or landmark index
    gives NaN (the kernel checks the index before any load), too many cameras is rejected;
  * the property the entry point exists for: repeated calls on a large problem leave the
    device's free memory unchanged.
This file is collected last on purpose."""
import numpy as np
import pytest

import bal_synth
from oracle import camera_model as cm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def poba():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as m
    m.library()
    return m


def _dev(a, dt):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()


def _noalloc(poba, cams, lms, obs, ci, li, w, stream):
    import torch
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        poba.ba_cost_noalloc(cams, lms, obs, ci, li, out, weights=w, stream=stream)
    stream.synchronize()
    return float(out.item())


def _noalloc_problem(poba, p, stream, cam_idx=None, lm_idx=None):
    import torch
    ci = p.cam_idx if cam_idx is None else cam_idx
    li = p.lm_idx if lm_idx is None else lm_idx
    return _noalloc(poba, _dev(p.cams0, torch.float64), _dev(p.lms0, torch.float64),
                    _dev(p.obs, torch.float64), _dev(ci, torch.int32), _dev(li, torch.int32),
                    None if p.weights is None else _dev(p.weights, torch.float64), stream)


def _handle_cost(poba, p):
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    try:
        return poba.ba_cost(h)
    finally:
        poba.ba_destroy(h)


def _oracle_cost(p):
    return cm.cost(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)


def test_noalloc_cost_matches_oracle_twice_in_a_row(poba):
    import torch
    s = torch.cuda.Stream()
    problems = [bal_synth.make_problem(60, 3000, track=("uniform", 3, 4), visibility="clustered", seed=201),
                bal_synth.make_problem(17, 500, track=("uniform", 2, 6), weighted=True, seed=202)]
    for p in problems:
        got, ref = _noalloc_problem(poba, p, s), _oracle_cost(p)
        assert np.isfinite(got)
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
        hc = _handle_cost(poba, p)
        assert abs(got - hc) <= 1e-12 * hc, (got, hc)
    # the same problem again after a different one: no state leaks between calls
    got, ref = _noalloc_problem(poba, problems[0], s), _oracle_cost(problems[0])
    assert abs(got - ref) <= 1e-12 * ref


def test_noalloc_empty_observations_give_zero(poba):
    import torch
    s = torch.cuda.Stream()
    cams = _dev(np.tile([0, 0, 0, 0, 0, -5, 500, 0, 0], (3, 1)), torch.float64)
    lms = _dev(np.zeros((2, 3)), torch.float64)
    obs = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    idx = torch.zeros((0,), dtype=torch.int32, device="cuda")
    assert _noalloc(poba, cams, lms, obs, idx, idx, None, s) == 0.0


@pytest.mark.parametrize("which", ["lm_high", "lm_negative", "cam_high"])
def test_noalloc_out_of_range_index_gives_nan(poba, which):
    import torch
    s = torch.cuda.Stream()
    p = bal_synth.make_problem(12, 400, track=("uniform", 2, 4), seed=203)
    ci, li = p.cam_idx.copy(), p.lm_idx.copy()
    k = p.n_obs // 2
    if which == "lm_high":
        li[k] = p.n_lms
    elif which == "lm_negative":
        li[k] = -1
    else:
        ci[k] = p.n_cams
    assert np.isnan(_noalloc_problem(poba, p, s, cam_idx=ci, lm_idx=li))
    # the scratch is whole afterwards: the valid problem gives the oracle's cost again
    got, ref = _noalloc_problem(poba, p, s), _oracle_cost(p)
    assert abs(got - ref) <= 1e-12 * ref


def test_noalloc_leaves_device_memory_unchanged(poba):
    """After one warm-up call (which loads the module), further calls on a 1,000,000-observation
    problem change neither the device's free memory nor torch's allocation counters."""
    import torch
    s = torch.cuda.Stream()
    p = bal_synth.make_problem(2000, 250000, track=("uniform", 3, 5), visibility="clustered",
                               seed=204)
    args = (_dev(p.cams0, torch.float64), _dev(p.lms0, torch.float64), _dev(p.obs, torch.float64),
            _dev(p.cam_idx, torch.int32), _dev(p.lm_idx, torch.int32))
    outs = torch.zeros((6,), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        poba.ba_cost_noalloc(*args, outs[5:6], stream=s)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    with torch.cuda.stream(s):
        for i in range(5):
            poba.ba_cost_noalloc(*args, outs[i:i + 1], stream=s)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    ref = _oracle_cost(p)
    for v in outs.cpu().numpy():
        assert abs(float(v) - ref) <= 1e-12 * ref


def test_noalloc_rejects_more_cameras_than_its_scratch_holds(poba):
    import torch
    n = poba.BA_NOALLOC_MAX_CAMS + 1
    cams = torch.zeros((n, 9), dtype=torch.float64, device="cuda")
    lms = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    obs = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    idx = torch.zeros((0,), dtype=torch.int32, device="cuda")
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(poba.PobaError) as e:
        poba.ba_cost_noalloc(cams, lms, obs, idx, idx, out)
    assert e.value.status_name == "BA_ERR_INVALID_ARG"
    assert "4096" in str(e.value)
