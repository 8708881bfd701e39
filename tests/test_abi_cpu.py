"""The C-ABI library builds, loads and exports every symbol include/poba.h declares; argument
validation that runs before any CUDA call is checked here without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "poba.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2204_12834_gb300 import build as b
    b.build()
    import paper_2204_12834_gb300 as poba
    return poba.library()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("ba_create", "ba_linearize", "ba_solve_schur_power", "ba_lm_step", "ba_cost",
                 "ba_get_params", "ba_get_step", "ba_destroy", "ba_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2204_12834_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_status_strings_and_defaults(lib):
    assert lib.ba_status_string(0) == b"BA_OK"
    assert lib.ba_status_string(4) == b"BA_ERR_NOT_SPD"
    import paper_2204_12834_gb300 as poba
    o = poba.ba_default_options()
    # Sec. 5.1: lambda0 1e-4, 50 LM iterations, func tol 1e-6, 20 inner iterations, eps 0.01
    assert (o.lambda0, o.func_tol, o.eps, o.max_lm, o.max_inner) == (1e-4, 1e-6, 0.01, 50, 20)


def _desc(n_c=3, n_l=4, n_o=6, seed=0):
    rng = np.random.default_rng(seed)
    cams = rng.normal(size=(n_c, 9))
    lms = rng.normal(size=(n_l, 3))
    obs = rng.normal(size=(n_o, 2))
    ci = rng.integers(0, n_c, n_o).astype(np.int32)
    li = rng.integers(0, n_l, n_o).astype(np.int32)
    return cams, lms, obs, ci, li


@pytest.mark.parametrize("case", ["bad_cam_index", "bad_lm_index", "zero_cams", "nan_obs",
                                  "neg_weight", "bad_precision"])
def test_create_rejects_bad_inputs_before_touching_the_gpu(lib, case):
    import paper_2204_12834_gb300 as poba
    cams, lms, obs, ci, li = _desc()
    w = None
    prec = poba.BA_FP64
    expect = "BA_ERR_INVALID_ARG"
    if case == "bad_cam_index":
        ci[2] = 3
    elif case == "bad_lm_index":
        li[0] = -1
    elif case == "zero_cams":
        cams = cams[:0]
    elif case == "nan_obs":
        obs[1, 0] = np.nan
        expect = "BA_ERR_NONFINITE"
    elif case == "neg_weight":
        w = np.ones(obs.shape[0])
        w[3] = -1.0
    elif case == "bad_precision":
        prec = 7
    with pytest.raises(poba.PobaError) as e:
        poba.ba_create(cams, lms, obs, ci, li, weights=w, precision=prec)
    assert e.value.status_name == expect, str(e.value)


def test_bad_options_rejected(lib):
    import paper_2204_12834_gb300 as poba
    cams, lms, obs, ci, li = _desc()
    for kw in (dict(lambda0=0.0), dict(eps=-1.0), dict(max_inner=-1), dict(damping_mode=3)):
        with pytest.raises(poba.PobaError) as e:
            poba.ba_create(cams, lms, obs, ci, li, options=poba.ba_default_options(**kw))
        assert e.value.status_name == "BA_ERR_INVALID_ARG"


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.ba_linearize(None, None) == 1
    assert lib.ba_lm_step(None, None) == 1
    assert lib.ba_destroy(None) == 0


def test_noalloc_cost_rejects_bad_arguments_before_any_cuda_call(lib):
    """ba_cost_noalloc checks sizes, its scratch limit, NULL pointers and the 16-byte alignment
    of obs on the host, before it asks CUDA for anything; the pointers here are never read."""
    import ctypes as C
    from paper_2204_12834_gb300 import BA_NOALLOC_MAX_CAMS
    fake = C.c_void_p(0x10000)            # aligned, never dereferenced
    odd = C.c_void_p(0x10008)             # 8 mod 16
    cases = [
        ((0, 1, 0, fake, fake, fake, fake, fake, None, fake), "n_cams >= 1"),
        ((1, 0, 0, fake, fake, fake, fake, fake, None, fake), "n_lms >= 1"),
        ((1, 1, -1, fake, fake, fake, fake, fake, None, fake), "n_obs >= 0"),
        ((BA_NOALLOC_MAX_CAMS + 1, 1, 0, fake, fake, fake, fake, fake, None, fake),
         str(BA_NOALLOC_MAX_CAMS)),
        ((1, 1, 0, None, fake, fake, fake, fake, None, fake), "NULL"),
        ((1, 1, 0, fake, fake, fake, fake, fake, None, None), "NULL"),
        ((1, 1, 4, fake, fake, None, fake, fake, None, fake), "NULL observation"),
        ((1, 1, 4, fake, fake, odd, fake, fake, None, fake), "16-byte aligned"),
    ]
    for args, words in cases:
        assert lib.ba_cost_noalloc(*args, None) == 1, args  # BA_ERR_INVALID_ARG
        assert words in lib.ba_last_error().decode(), (args, lib.ba_last_error())


def test_create_batch_rejects_bad_problems_before_touching_the_gpu(lib):
    """ba_create_batch validates every problem on the host: an empty batch, mixed precisions
    and a bad index in one problem are rejected, the last naming the problem."""
    import ctypes as C
    import paper_2204_12834_gb300 as poba
    from paper_2204_12834_gb300._lib import ProblemDesc
    ok = _desc(seed=1)
    bad = list(_desc(seed=2))
    bad[3] = bad[3].copy()
    bad[3][4] = 3  # camera index == n_cams
    with pytest.raises(poba.PobaError) as e:
        poba.ba_create_batch([ok, tuple(bad)])
    assert e.value.status_name == "BA_ERR_INVALID_ARG"
    assert "problem 1: cam_idx[4] out of range" in str(e.value)

    keep = []
    descs = (ProblemDesc * 2)()
    for i, (pr, prec) in enumerate(((ok, poba.BA_FP64), (_desc(seed=3), poba.BA_FP32_BULK))):
        poba._fill_desc(descs[i], *pr, None, prec, None, keep)
    out = C.c_void_p()
    opts = poba.ba_default_options()
    assert lib.ba_create_batch(descs, 2, C.byref(opts), C.byref(out)) == 1
    assert "same precision" in lib.ba_last_error().decode()
    assert not out.value
    assert lib.ba_create_batch(descs, 0, C.byref(opts), C.byref(out)) == 1
    assert "n_problems must be >= 1" in lib.ba_last_error().decode()
