"""Writes tests/golden/lm_direct_<workload>.json: the oracle's Levenberg-Marquardt run to
convergence with the exact solve of the reduced camera system on one seeded workload.  Test
infrastructure: it calls only `oracle/` and the seeded generator.

The run uses the settings of Sec. 5.1: starting damping 1e-4, a relative function tolerance of
1e-6 and at most 50 iterations. Each step is an exact solve of S dx_p = -b~ (explicit
block-sparse S, Schur-Jacobi PCG to a relative residual of 1e-12) in place of the truncated
series. Its final cost is one of the solvers' final objectives from which the performance
profiles of Sec. 5 take f* (the lowest final objective of any solver on the problem). The
time-to-cost threshold is then f_tau = f* + tau (f0 - f*).

Usage: python tests/golden/make_lm_direct_reference.py [workload]   (default: the clustered
1200-camera problem; about 15 oracle iterations, a few minutes single-threaded)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bal_synth  # noqa: E402
from oracle import camera_model as cm  # noqa: E402
from oracle import lm as olm  # noqa: E402


def main(workload="clustered_1200c_160000l"):
    p = bal_synth.preset(workload)
    args = (p.obs, p.cam_idx, p.lm_idx, p.weights)
    f0 = float(cm.cost(p.cams0, p.lms0, *args))
    opts = olm.Options(lambda0=1e-4, func_tol=1e-6, max_lm=50)
    t0 = time.perf_counter()
    cams, lms, hist = olm.lm_solve(p, opts, solver="direct")
    seconds = time.perf_counter() - t0
    final = float(cm.cost(cams, lms, *args))
    out = {
        "workload": workload,
        "n_cams": int(p.n_cams), "n_lms": int(p.n_lms), "n_obs": int(p.n_obs),
        "solver": "oracle LM, exact reduced solve (explicit block-sparse S, Schur-Jacobi PCG "
                  "to 1e-12)",
        "settings": {"lambda0": opts.lambda0, "func_tol": opts.func_tol, "max_lm": opts.max_lm},
        "initial_cost": f0,
        "final_cost": final,
        "iterations": len(hist),
        "accepted": int(sum(h["accepted"] for h in hist)),
        # the relative function tolerance fired on the last (accepted) step
        "converged": bool(hist[-1]["accepted"] and (hist[-1]["cost_before"] - hist[-1]["cost_after"])
                          / hist[-1]["cost_before"] < opts.func_tol),
        "oracle_seconds": round(seconds, 1),
    }
    path = os.path.join(HERE, f"lm_direct_{workload}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out))


if __name__ == "__main__":
    main(*sys.argv[1:])
