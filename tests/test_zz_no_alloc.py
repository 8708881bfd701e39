"""The allocation-free cost entry point (ba_cost_noalloc) against the handle-based ba_cost.

ba_cost_noalloc serves callers that must not let a library allocate device memory (cudaMalloc
and cudaFree synchronise the device; some processes hand all device memory to one allocator).
It keeps its scratch in one fixed device array shared by all calls, so this test makes two
calls in a row on different problems and checks each against ba_cost (float64, 1e-12
relative), then the size limit.  This file is collected last on purpose."""
import numpy as np
import pytest

import bal_synth

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


def _cost_both(poba, p, stream):
    import torch
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).cuda()
    cams, lms = dev(p.cams0, torch.float64), dev(p.lms0, torch.float64)
    obs = dev(p.obs, torch.float64)
    ci, li = dev(p.cam_idx, torch.int32), dev(p.lm_idx, torch.int32)
    w = None if p.weights is None else dev(p.weights, torch.float64)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        poba.ba_cost_noalloc(cams, lms, obs, ci, li, out, weights=w, stream=stream)
    stream.synchronize()
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    ref = poba.ba_cost(h)
    poba.ba_destroy(h)
    return float(out.item()), ref


def test_noalloc_cost_matches_ba_cost_twice_in_a_row(poba):
    import torch
    s = torch.cuda.Stream()
    problems = [bal_synth.make_problem(60, 3000, track=("uniform", 3, 4), visibility="clustered", seed=201),
                bal_synth.make_problem(17, 500, track=("uniform", 2, 6), weighted=True, seed=202)]
    for p in problems:
        got, ref = _cost_both(poba, p, s)
        assert np.isfinite(got)
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)
    # the same problem again after a different one: no state leaks between calls
    got, ref = _cost_both(poba, problems[0], s)
    assert abs(got - ref) <= 1e-12 * ref


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
