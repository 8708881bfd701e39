"""bench.py's CPU-baseline leg (host only): the single-threaded oracle LM with the power-series
solve, the same LM with the oracle's exact reduced solve, and independent single-threaded
replicas on every host core, each reporting its iteration rate and peak resident set."""
import bench


def test_cpu_baseline_reports_every_leg():
    args = bench.parse_args(["--workload", "uniform_16c_1000l", "--cpu-seconds", "0.2"])
    line = bench.cpu_baseline(args)
    assert line["kind"] == "oracle" and line["cores"] == 1
    assert line["value"] > 0 and line["unit"] == "LM iterations/s"
    assert line["peak_rss_bytes"] > 10 << 20
    d = line["direct"]
    assert d["value"] > 0 and d["cores"] == 1 and "PCG" in d["solver"]
    a = line["all_cores"]
    assert a["value"] > 0 and 1 <= a["cores"] <= a["host_cores"] == bench.host_cores()
    assert a["peak_rss_bytes_per_replica"] > 10 << 20
    assert str(a["cores"]) in a["sample"]


def test_oracle_workers_start_together():
    """Replicas wait at a file barrier after building the problem, so their timed windows
    overlap: every start precedes every end."""
    args = bench.parse_args(["--workload", "uniform_16c_1000l"])
    reps = bench.run_oracle_workers(args, "power", 0.3, 3)
    assert len(reps) == 3 and all(r["iters"] >= 1 for r in reps)
    assert max(r["start"] for r in reps) < min(r["end"] for r in reps)
