"""The debug build (libpoba_checks.so, compiled with -DPOBA_CHECKS): every camera, landmark,
slot, position and segment index the kernels read from the schedule is checked before use, and
every sub-buffer of a handle's device allocations is followed by guard bytes.  Each call that
synchronises verifies the check record and the guards and raises BA_ERR_CHECK on a failure.

The parity, edge-case and long-track GPU suites run through the debug build in a child process
(POBA_CHECKS=1 makes the binding load it); a short script there also asserts that the record is
clean after LM steps in every series form and in a batch."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CLEAN_SCRIPT = r"""
import numpy as np
import bal_synth
import paper_2204_12834_gb300 as poba
assert poba.library()._name.endswith("libpoba_checks.so")
p = bal_synth.make_problem(300, 3000, track=("long", 2, 6, (400,)), visibility="clustered", seed=7)
for prec in (0, 1):
    for form in (0, 1, 3, 4, 5):
        h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, precision=prec,
                           options=poba.ba_default_options(series_exec=form))
        for _ in range(3):
            poba.ba_lm_step(h)
        r = poba.ba_debug_checks(h)
        assert r["enabled"] and r["site"] == 0 and r["count"] == 0, (prec, form, r)
        poba.ba_destroy(h)
hb = poba.batch_from_problems(bal_synth.make_batch(12), precision=1)
for _ in range(3):
    poba.ba_lm_step_batch(hb)
r = poba.ba_debug_checks(hb)
assert r["enabled"] and r["site"] == 0, r
print("clean")
"""


@pytest.fixture(scope="module")
def checks_env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2204_12834_gb300 import build as b
    b.build()
    b.build(checks=True)
    env = dict(os.environ, POBA_CHECKS="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    return env


def test_release_build_reports_checks_disabled():
    import bal_synth
    import paper_2204_12834_gb300 as poba
    from paper_2204_12834_gb300 import build as b
    b.build()
    p = bal_synth.make_problem(8, 100, seed=3)
    h = poba.ba_create(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx)
    r = poba.ba_debug_checks(h)
    assert r == {"enabled": False, "site": 0, "count": 0, "index": 0}


def test_checked_build_record_stays_clean(checks_env):
    out = subprocess.run([sys.executable, "-c", CLEAN_SCRIPT], cwd=ROOT, env=checks_env,
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0 and "clean" in out.stdout, out.stdout[-2000:] + out.stderr[-3000:]


def test_checked_build_runs_the_parity_suites(checks_env):
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_gpu_edge.py", "tests/test_gpu_long_tracks.py"]
    out = subprocess.run(cmd, cwd=ROOT, env=checks_env, capture_output=True, text=True,
                         timeout=2400)
    assert out.returncode == 0, out.stdout[-4000:] + out.stderr[-2000:]
