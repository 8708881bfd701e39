"""bench.py's reference arm on the host (no GPU): the FP64 oracle timed on a small workload
prints one JSON line with the keys of the bench contract, and under a multi-rank launch every
rank but 0 exits 0 without work or output."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    env.pop("POBA_REFERENCE_CHILD", None)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "uniform_16c_1000l", "--steps", "3", "--warmup", "3"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    p = _run()
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["steps"] == 3 and d["higher_is_better"] is True
    assert d["warmup"] == 3  # --warmup is honoured in full
    assert d["unit"] == "LM iterations/s" and d["dtype"] == "f64"
    assert d["config"]["workload"] == "uniform_16c_1000l"
    assert d["config"]["n_cams"] == 16 and d["config"]["n_lms"] == 1000
    assert "no BAL counterpart" in d["data"]
    # the same config dict as the library arm's line (built by the same function)
    sys.path.insert(0, ROOT)
    import bal_synth
    import bench
    assert d["config"] == json.loads(json.dumps(bench.headline_config(
        "uniform_16c_1000l", bal_synth.preset("uniform_16c_1000l"), 1)))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_data_note_names_the_stand_in():
    sys.path.insert(0, ROOT)
    import bench
    assert "Ladybug-1197" in bench.data_note("clustered_1200c_160000l")
    assert "Venice-1778" in bench.data_note("powerlaw_10000c_1000000l")
    assert "synthetic" in bench.data_note("weighted_200c_20000l")


def test_oracle_lm_iterations_restart_and_count():
    """The reference arm's step loop runs exactly n oracle LM iterations, restarting from x0
    after a solve converges (so n may exceed one solve's length)."""
    sys.path.insert(0, ROOT)
    import bal_synth
    import bench
    from oracle import lm as olm
    p = bal_synth.preset("uniform_16c_1000l")
    _, _, hist = olm.lm_solve(p)
    one = len(hist)
    assert one < 50  # this small problem converges
    n = one + 3
    assert bench.oracle_lm_iterations(p, n) == n
