"""The stored final cost of the oracle's LM with the exact reduced solve
(tests/golden/lm_direct_clustered_1200c_160000l.json, written by make_lm_direct_reference.py),
which bench.py folds into f* of the time-to-cost threshold (Sec. 5, performance profiles).
It is pinned here to the problem it was made for (sizes and initial cost from the generator
and the oracle's cost), to convergence under the Sec. 5.1 settings, and to the chi-square noise
floor of a converged solve: E[F*] = (2 n_o - (9 n_c + 3 n_l - 7)) sigma^2 / 2, standard
deviation sqrt(dof / 2), with sigma = 1 px of injected noise."""
import json
import math
import os

import pytest

import bal_synth
import bench
from oracle import camera_model as cm

WORKLOAD = "clustered_1200c_160000l"
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    f"lm_direct_{WORKLOAD}.json")


@pytest.fixture(scope="module")
def stored():
    with open(PATH) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def problem():
    return bal_synth.preset(WORKLOAD)


def test_made_for_this_problem(stored, problem):
    p = problem
    assert (stored["n_cams"], stored["n_lms"], stored["n_obs"]) == (p.n_cams, p.n_lms, p.n_obs)
    f0 = cm.cost(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
    assert abs(stored["initial_cost"] - f0) <= 1e-12 * f0
    assert stored["settings"] == {"lambda0": 1e-4, "func_tol": 1e-6, "max_lm": 50}


def test_converged_at_the_noise_floor(stored, problem):
    p = problem
    assert stored["converged"] and stored["iterations"] < 50
    dof = 2 * p.n_obs - (9 * p.n_cams + 3 * p.n_lms - 7)
    mean, sd = dof / 2.0, math.sqrt(dof / 2.0)
    assert abs(stored["final_cost"] - mean) < 5 * sd


def test_bench_uses_it_only_for_its_problem(stored, problem):
    f0 = stored["initial_cost"]
    assert bench.oracle_direct_final(WORKLOAD, problem, f0) == stored["final_cost"]
    assert bench.oracle_direct_final(WORKLOAD, problem, f0 * (1 + 1e-6)) is None
    other = bal_synth.preset("uniform_16c_1000l")
    assert bench.oracle_direct_final(WORKLOAD, other, f0) is None
    assert bench.oracle_direct_final("uniform_16c_1000l", problem, f0) is None
