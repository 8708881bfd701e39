#!/usr/bin/env python
"""Benchmark of GPU Power Bundle Adjustment (LM iterations/s on one GB300).

A step is one Levenberg-Marquardt iteration of the whole hot path: linearise (residuals,
Jacobians, U / V / b blocks), damp and invert the blocks, form b~ and x(0), run the power
series with the stop rule (eps 0.01, at most 20 terms), back-substitute, evaluate F(x + dx)
and the model decrease, accept / reject and update lambda.  Consecutive steps run real LM solves
from the initial state: a solve runs until the relative function tolerance (1e-6) is met or 50
iterations have passed, then the state is reset to x0 outside the timed events.  The L2 cache is
flushed (512 MiB write) before every timed step; each step is timed with CUDA events on the
library's stream.

Output: one JSON line (rank 0).  `value` is LM iterations/s summed over ranks (each rank solves
its own replica of the problem; no collective on the data path).  Extra keys report series
solves/s, time to the tau = 1% cost threshold, the roofline of the dominant kernel, the
float32-bulk variant, an end-to-end number through the public API with host buffers, and the
FP64 CPU oracle timed on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl poba|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bal_synth  # noqa: E402

WORKLOAD = "clustered_1200c_160000l"
METRIC = "LM iterations/s (power-series Schur PoBA, BAL camera model)"
L2_FLUSH_BYTES = 512 << 20
# FP64 FMA issue rate of one GB300 SM per clock; ba_probe_fp64_fma (bench.py --fp64-probe)
# measures the device rate that backs it
FP64_FMA_PER_CLK_PER_SM = 2
DEFAULT_MAX_SM_MHZ = 2070.0
REFERENCE_BUDGET_S = 240.0
FALLBACK_HBM_GBS = 6800.0


# the BAL problem each seeded synthetic workload stands in for (sizes only; no BAL data is read)
STANDS_IN_FOR = {
    "clustered_1200c_160000l": "BAL Ladybug-1197",
    "powerlaw_10000c_1000000l": "BAL Venice-1778",
}


def fp64_peak_tflops(sms: int, max_mhz) -> float:
    """Derived FP64 FMA peak: SMs x FMA/clk/SM x 2 FLOP x maximum SM clock (the sampled
    clocks.max.sm, else GB300's 2070 MHz)."""
    return sms * FP64_FMA_PER_CLK_PER_SM * 2 * float(max_mhz or DEFAULT_MAX_SM_MHZ) * 1e6 / 1e12


def headline_config(workload: str, p, world: int) -> dict:
    """The `config` of the headline line; both arms print the same one."""
    return {"workload": workload, "n_cams": p.n_cams, "n_lms": p.n_lms, "n_obs": p.n_obs,
            "role": ("headline: the plain vs FP32-bulk PoBA problem (1,200 cameras, 160,000 "
                     "landmarks, ~560,000 observations, 3-4 per landmark, clustered visibility), "
                     "the workload on which the metric's time to 1% cost and the FP32-vs-FP64 "
                     "error are defined; `value` is its FP64 LM iterations/s, `fp32_bulk` the "
                     "FP32-bulk form; the 10,000-camera power-law problem is under `large`"),
            "visibility": "clustered window 8, tracks U{3,4}",
            "series": {"eps": 0.01, "max_inner": 20},
            "lm": {"lambda0": 1e-4, "func_tol": 1e-6, "max_lm": 50, "restart_from_x0": True},
            "l2": "GPU arm: flushed before every timed step (512 MiB write)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def data_note(workload: str) -> str:
    what = STANDS_IN_FOR.get(workload)
    tail = f"stands in for {what}" if what else "no BAL counterpart"
    return f"synthetic (seeded BAL-model problem; {tail})"


# ---------------------------------------------------------------------------------------
def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["poba", "reference"], default="poba")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-sub-problems section (256 problems, FP32 bulk)")
    ap.add_argument("--batch-solves", type=int, default=3)
    ap.add_argument("--no-pcg", action="store_true",
                    help="skip the PCG comparison (Schur-Jacobi and power-series preconditioners)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large single-problem section (10,000 cameras, 5M observations)")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the adjoint section (200 cameras, 20,000 landmarks, weighted)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-baseline-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-solver", choices=["power", "direct"], default="power",
                    help=argparse.SUPPRESS)
    ap.add_argument("--cpu-sync-dir", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-sync-n", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--fp64-probe", action="store_true",
                    help="only measure the device's FP64 FMA rate (ba_probe_fp64_fma) with the "
                         "SM clocks sampled during it, and print one JSON line")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run only this many untimed LM steps (for ncu captures)")
    ap.add_argument("--profile-precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--profile-form", type=int, default=0,
                    help="profile mode: the series form to run (ba_set_schedule series_exec; "
                         "0 keeps the handle's default)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="profile mode on the 256-problem batch instead of the single problem")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_max(v: float, device=None) -> float:
    """Max of a scalar over all ranks (identity when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, slowest_seconds: float) -> float:
    """Units processed by all ranks / the slowest rank's time (weak scaling: every rank solves
    its own replica, so the job rate is world x units / max time)."""
    return world * units_per_rank / slowest_seconds


# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling (200 ms) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="poba_clocks_", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def measured_peaks() -> tuple[float, str, float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured", float(d.get("bf16_tflops", 0.0)), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback", 1900.0, "fallback"


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in ("kernels_persistent.cu", "series_body.cuh", "tile_common.cuh", "poba_internal.cuh",
              "jacobian_io.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2204_12834_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(precision: str, form: int, workload: str = WORKLOAD):
    """DRAM bytes per series term of the persistent kernel in the given form (3 plain, 4 staged,
    5 dataflow) on `workload`, from the committed ncu summary, if the kernel source is unchanged
    since the capture and that form was captured; else None."""
    path = os.path.join(ROOT, "profiles", f"series_persistent_{workload}.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_source_sha") != kernel_source_sha():
        return None
    # an entry per captured form: "<precision>" and "<precision>_form<k>"
    for e in (d.get(precision, {}), d.get(f"{precision}_form{form}", {})):
        if e.get("form") == form:
            return e.get("dram_bytes_per_term")
    return None


def step_stats(ms) -> dict:
    """Median and spread of the per-step CUDA-event times (steps differ: a rejected step skips
    the linearisation, and the series stops after a varying number of terms)."""
    a = np.asarray(ms, dtype=np.float64)
    if a.size == 0:
        return {"median": None, "p10": None, "p90": None, "n": 0}
    return {"median": float(np.median(a)), "p10": float(np.percentile(a, 10)),
            "p90": float(np.percentile(a, 90)), "n": int(a.size)}


def oracle_direct_final(workload: str, p, f0_gpu: float):
    """Final cost of the oracle's LM with the exact reduced solve, run to convergence from x0
    (stored by tests/golden/make_lm_direct_reference.py), if it was made for this problem: the
    same sizes and an initial cost equal to the library's to 1e-9.  One of the solvers' final
    objectives from which f* of the time-to-cost threshold is taken (Sec. 5, performance
    profiles)."""
    path = os.path.join(ROOT, "tests", "golden", f"lm_direct_{workload}.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if (d.get("n_cams"), d.get("n_lms"), d.get("n_obs")) != (p.n_cams, p.n_lms, p.n_obs):
        return None
    if abs(d["initial_cost"] - f0_gpu) > 1e-9 * abs(f0_gpu) or not d.get("converged"):
        return None
    return float(d["final_cost"])


# ---------------------------------------------------------------------------------------
def series_term_units(p, s: int):
    """Algorithmic (minimal) bytes and flops of one power-series term
    t_i = U^-1 W V^-1 W^T t_{i-1} applied matrix-free, per Sec. 4.3: per observation J_p and
    J_l (24 s) and its camera index (4 B), 48 FMA (J_p t 18, J_l^T u 6, J_l z 6, J_p^T w 18);
    per landmark V^-1 (6 s) and its segment offset (4 B), 9 FMA; per camera U^-1 (45 x 8 B)
    and t, x read and written (27 x 8 B), 81 FMA."""
    n_o, n_l, n_c = p.n_obs, p.n_lms, p.n_cams
    bytes_ = n_o * (24 * s + 4) + n_l * (6 * s + 4) + n_c * (45 * 8 + 27 * 8)
    flops = n_o * 2 * 48 + n_l * 2 * 9 + n_c * 2 * 81
    return bytes_, flops


def series_term_design_bytes(p, group_slots: int, s: int) -> int:
    """Bytes one term moves in this design: per observation J (24 s) and its 4-byte chunk code;
    per landmark V^-1 (6 s) and its 2-byte segment offset; per group slot (one per group and
    camera it touches, ba_get_schedule's n_group_slots) the current term gathered (12 s), the
    9-vector partial written and read back (2 x 9 s); per camera U^-1 (81 x 8 B), x read and
    written and the new term (12 s)."""
    n_o, n_l, n_c = p.n_obs, p.n_lms, p.n_cams
    return (n_o * (24 * s + 4) + n_l * (6 * s + 2) + group_slots * 30 * s
            + n_c * (81 * 8 + 18 * 8 + 12 * s))


def explicit_s_bytes(p) -> int:
    """Block-sparse explicit S (what an explicit-Schur PCG stores): distinct camera pairs that
    share a landmark (upper triangle incl. diagonal) x 81 doubles.  Landmarks are grouped by
    track length so that each group's pairs come from one index table."""
    order = np.lexsort((p.cam_idx, p.lm_idx))
    cams = p.cam_idx[order].astype(np.int64)
    counts = np.bincount(p.lm_idx, minlength=p.n_lms)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    nc = p.n_cams
    codes = []
    for k in np.unique(counts[counts > 0]):
        ls = starts[counts == k]
        tracks = cams[ls[:, None] + np.arange(k)[None, :]]  # [n_k, k] sorted cameras
        i, j = np.triu_indices(int(k))
        codes.append((tracks[:, i] * nc + tracks[:, j]).ravel())
    if not codes:
        return 0
    return int(np.unique(np.concatenate(codes)).size) * 81 * 8


# ---------------------------------------------------------------------------------------
def run_poba(args):
    import torch
    import paper_2204_12834_gb300 as poba
    from paper_2204_12834_gb300 import build as pbuild

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    pbuild.build()
    poba.library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    p = bal_synth.preset(args.workload)
    to_dev = lambda a: torch.as_tensor(a).to(dev)

    def make(precision, **opt):
        with torch.cuda.stream(stream):
            return poba.ba_create(to_dev(p.cams0), to_dev(p.lms0), to_dev(p.obs), to_dev(p.cam_idx),
                                  to_dev(p.lm_idx), None if p.weights is None else to_dev(p.weights),
                                  precision=precision, options=poba.ba_default_options(**opt),
                                  stream=stream)

    cams0_d, lms0_d = to_dev(p.cams0), to_dev(p.lms0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    if args.profile_steps:
        prec = poba.BA_FP64 if args.profile_precision == "fp64" else poba.BA_FP32_BULK
        if args.profile_batch:
            hb = poba.batch_from_problems(bal_synth.make_batch(256), precision=prec, stream=stream)
            if args.profile_form:
                poba.ba_set_schedule(hb, series_exec=args.profile_form)
            for _ in range(args.profile_steps):
                poba.ba_lm_step_batch(hb)
        else:
            h = make(prec)
            if args.profile_form:
                poba.ba_set_schedule(h, series_exec=args.profile_form)
            for _ in range(args.profile_steps):
                poba.ba_lm_step(h)
        torch.cuda.synchronize()
        return

    def reset(h):
        poba.ba_set_params(h, cams0_d, lms0_d)
        poba.ba_set_lm_state(h, 1e-4, 2.0, 0)

    def lm_block(h, n_steps, timed):
        """n_steps LM iterations (restarting from x0 after convergence / 50 iterations)."""
        evs = []
        n_lin = 0
        iters_in_solve = 0
        with torch.cuda.stream(stream):
            for _ in range(n_steps):
                if iters_in_solve >= 50:
                    reset(h)
                    iters_in_solve = 0
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s = poba.ba_lm_step(h)
                e1.record(stream)
                evs.append((e0, e1))
                iters_in_solve += 1
                if s["converged"]:
                    iters_in_solve = 50
        stream.synchronize()
        ms = [a.elapsed_time(b) for a, b in evs]
        return ms

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return dist_max(v, dev)

    results = {}
    clocks = ClockSampler(local)
    for name, prec in (("fp64", poba.BA_FP64), ("fp32_bulk", poba.BA_FP32_BULK)):
        h = make(prec)
        lm_block(h, args.warmup, False)
        tuned = poba.ba_autotune(h, trials=3)  # picks the series execution form (untimed)
        reset(h)
        poba.ba_set_timing(h, True)
        launches0 = poba.ba_kernel_launches(h)
        if name == "fp64":
            clocks.start()
        barrier()
        ms = lm_block(h, args.steps, True)
        barrier()
        if name == "fp32_bulk":
            clk = clocks.stop()
        launches = poba.ba_kernel_launches(h) - launches0
        total_ms = max_over_ranks(sum(ms))
        timing = poba.ba_get_timing(h)
        poba.ba_set_timing(h, False)
        results[name] = dict(h=h, ms=ms, total_ms=total_ms, timing=timing, launches=launches,
                             tuned=tuned)

    # series solves/s at the current linearisation of each handle
    for name, r in results.items():
        h = r["h"]
        poba.ba_linearize(h, want_cost=False)
        evs = []
        infos = []
        n = max(10, min(args.steps, 200))
        with torch.cuda.stream(stream):
            for _ in range(n):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                infos.append(poba.ba_solve_schur_power(h, 1e-4))
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        sms = sum(a.elapsed_time(b) for a, b in evs)
        r["solves_per_s"] = world * n / (max_over_ranks(sms) / 1e3)
        r["solve_inner_mean"] = float(np.mean([i["inner_iters"] for i in infos]))

    # time to reach f_tau = f* + 0.01 (f0 - f*) in a fresh solve from x0 (per precision)
    traj = {}
    for name, prec in (("fp64", poba.BA_FP64), ("fp32_bulk", poba.BA_FP32_BULK)):
        h = make(prec)
        f0 = poba.ba_cost(h)
        t = 0.0
        pts = []
        with torch.cuda.stream(stream):
            for _ in range(50):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s = poba.ba_lm_step(h)
                e1.record(stream)
                stream.synchronize()
                t += e0.elapsed_time(e1) / 1e3
                pts.append((t, s["cost_after"] if s["accepted"] else s["cost_before"]))
                if s["converged"]:
                    break
        traj[name] = dict(f0=f0, pts=pts, final=pts[-1][1], iters=len(pts))
    f_star = min(v["final"] for v in traj.values())
    f_star_src = "lowest final cost of the GPU runs (FP64, FP32 bulk)"
    ref = oracle_direct_final(args.workload, p, traj["fp64"]["f0"])
    if ref is not None and ref < f_star:
        f_star, f_star_src = ref, "the oracle's direct-solve LM run to convergence"
    traj["fp64"]["f_star"] = {"value": f_star, "source": f_star_src, "oracle_direct_final": ref}
    for name, v in traj.items():
        f_tau = f_star + 0.01 * (v["f0"] - f_star)
        v["time_to_tau_s"] = next((t for t, c in v["pts"] if c <= f_tau), None)

    # end-to-end through the public API with host buffers: per step H2D of the state from
    # pinned host memory, one LM step, D2H of the new state into the other pinned pair, which
    # is the next step's input (the state crosses the host every step, with no host copy)
    h = make(poba.BA_FP64)
    pairs = [(torch.as_tensor(p.cams0).pin_memory(), torch.as_tensor(p.lms0).pin_memory())
             for _ in range(2)]
    views = [(c.numpy(), l.numpy()) for c, l in pairs]
    n_e2e = max(5, min(args.steps, 100))
    barrier()
    t0 = time.perf_counter()
    for i in range(n_e2e):
        src, dst = i % 2, (i + 1) % 2
        if i % 50 == 0:
            pairs[src][0].copy_(torch.as_tensor(p.cams0))
            pairs[src][1].copy_(torch.as_tensor(p.lms0))
            poba.ba_set_lm_state(h, 1e-4, 2.0, 0)
        poba.ba_set_params(h, pairs[src][0], pairs[src][1])
        poba.ba_lm_step(h)
        poba.ba_get_params(h, views[dst][0], views[dst][1])
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    state_bytes = (p.n_cams * 9 + p.n_lms * 3) * 8

    # roofline of the dominant kernel class
    hbm_peak, hbm_kind, _, _ = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    l2_bytes = getattr(props, "L2_cache_size", 0) or (126 << 20)
    max_mhz = float(clk.get("sm_max_mhz") or DEFAULT_MAX_SM_MHZ)
    peak64 = fp64_peak_tflops(sms, max_mhz)
    pr = max((poba.ba_probe_fp64_fma(4, 1 << 16, stream) for _ in range(3)),
             key=lambda d: d["flops_per_s"])
    probe = {"tflops": pr["flops_per_s"] / 1e12, "ms": pr["ms"],
             "what": "ba_probe_fp64_fma: 4 blocks/SM x 256 threads x 8 independent FMA chains, "
                     "best of 3 launches (untimed clocks; see bench.py --fp64-probe)"}

    def roofline(name):
        """Dominant kernel: the series (one term = tile phase and camera phase, plus the two
        grid barriers in a persistent form).  The timing classes count executed terms, so
        ms / count is the average time of one term."""
        r = results[name]
        cls = max(r["timing"], key=lambda k: r["timing"][k][0])
        ms_t, cnt = r["timing"]["series_tile"]
        ms_c, _ = r["timing"]["series_camera"]
        s = 8 if name == "fp64" else 4
        nb, nf = series_term_units(p, s)
        sched = poba.ba_get_schedule(r["h"])
        nd = series_term_design_bytes(p, sched["n_group_slots"], s)
        avg_s = (ms_t + ms_c) / 1e3 / max(cnt, 1)
        form = r["tuned"]["exec"]
        prec = "double" if name == "fp64" else "float"
        pair = (f"series_group_kernel<{prec}, 0> + camera_step_kernel<{prec}, 0> (one pair of "
                "launches per term")
        kernel = {0: pair + ")",
                  1: pair + ", inside the captured LM-step graph)",
                  3: f"series_persistent_kernel<{prec}> (one series term: group phase, camera "
                     "phase, two grid barriers)",
                  4: "series_staged_kernel (persistent; each chunk's inputs staged in shared "
                     "memory by bulk copies one chunk ahead; one term: group phase, camera "
                     "phase, two grid barriers)",
                  5: f"series_dataflow_kernel<{prec}> (persistent, no grid barriers: groups of "
                     "term i start once their cameras' term i-1 updates are published; one term "
                     "= the time of the whole launch / terms)"}.get(form, f"series form {form}")
        traffic = profiled_traffic(name, form)
        common = {"kernel": kernel, "series_form": r["tuned"], "schedule": sched,
                  "traffic": traffic, "algorithmic_bytes_per_term": nb,
                  "algorithmic_flops_per_term": nf, "design_bytes_per_term": nd,
                  "design_gbs": nd / avg_s / 1e9, "avg_term_us": avg_s * 1e6, "terms": cnt,
                  "dominant_class": cls}
        if name == "fp64":
            ach = nf / avg_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": peak64, "unit": "TFLOP/s",
                    "frac": ach / peak64,
                    "peak_kind": (f"derived FP64 FMA rate ({sms} SMs x {FP64_FMA_PER_CLK_PER_SM} "
                                  f"FMA/clk x 2 FLOP x {max_mhz:.0f} MHz max SM clock)"),
                    "fp64_probe": probe, "achieved_gbs": nb / avg_s / 1e9, **common}
        ach = nb / avg_s / 1e9
        line = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak,
                "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_kind == "measured"
                else "fallback 6800 GB/s",
                "achieved_tflops": nf / avg_s / 1e12, **common}
        if nb <= l2_bytes:
            # the float Jacobians of this problem fit in L2: after the first term of a solve
            # the series reads them from L2, so HBM does not bound it
            line["bound"] = "l2-resident"
            line["peak_kind"] += (f"; for comparison only: the term's {nb / 1e6:.0f} MB fit the "
                                  f"{l2_bytes / 1e6:.0f} MB L2, so DRAM is not its bound (the "
                                  "HBM-bound case is `large`)")
        return line

    batched = None if args.no_batch else batched_section(args, poba, torch, stream, dev,
                                                           max_over_ranks, barrier)

    adjoint = None if args.no_adjoint else adjoint_section(args, poba, torch, stream, dev)
    large = None if args.no_large else large_section(args, poba, torch, stream, dev,
                                                     max_over_ranks, barrier)
    pcg = None if args.no_pcg else pcg_section(poba, torch, stream, results)

    roof64 = roofline("fp64")
    roof32 = roofline("fp32_bulk")
    mem_gpu = poba.ba_memory_footprint(results["fp64"]["h"])
    mem_gpu32 = poba.ba_memory_footprint(results["fp32_bulk"]["h"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)

    if rank != 0:
        return
    r64, r32 = results["fp64"], results["fp32_bulk"]

    def kernel_avgs(r):
        return {k: {"avg_us": (v[0] * 1e3 / v[1]) if v[1] else None, "count": v[1],
                    "share": v[0] / max(sum(x[0] for x in r["timing"].values()), 1e-12)}
                for k, v in r["timing"].items()}

    line = {
        "metric": METRIC,
        "value": whole_job_rate(args.steps, world, r64["total_ms"] / 1e3),
        "unit": "LM iterations/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r64["total_ms"] / args.steps,
        "step_ms": step_stats(r64["ms"]),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": data_note(args.workload),
        "config": headline_config(args.workload, p, world),
        "roofline": roof64,
        "clocks": clk,
        "gpu_launches": int(r64["launches"]),
        "e2e": {"value": world * n_e2e / e2e_s, "unit": "LM iterations/s",
                "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
                "steps": n_e2e, "note": "ba_set_params (pinned host) + ba_lm_step + ba_get_params (host, into the other pinned pair: the next input)"},
        "solves_per_s": r64["solves_per_s"],
        "solve_inner_mean": r64["solve_inner_mean"],
        "time_to_1pct_cost_s": traj["fp64"]["time_to_tau_s"],
        "f_star": traj["fp64"]["f_star"],
        "lm_iters_to_converge": traj["fp64"]["iters"],
        "final_cost": traj["fp64"]["final"],
        "memory_bytes": mem_gpu,
        "explicit_S_bytes": explicit_s_bytes(p),
        "kernels": kernel_avgs(r64),
        "series_form": r64["tuned"],
        "fp32_bulk": {"value": whole_job_rate(args.steps, world, r32["total_ms"] / 1e3),
                      "unit": "LM iterations/s",
                      "ms_per_step": r32["total_ms"] / args.steps,
                      "step_ms": step_stats(r32["ms"]), "roofline": roof32,
                      "gpu_launches": int(r32["launches"]), "solves_per_s": r32["solves_per_s"],
                      "solve_inner_mean": r32["solve_inner_mean"],
                      "time_to_1pct_cost_s": traj["fp32_bulk"]["time_to_tau_s"],
                      "final_cost": traj["fp32_bulk"]["final"],
                      "final_cost_rel_to_fp64": traj["fp32_bulk"]["final"] / traj["fp64"]["final"] - 1.0,
                      "memory_bytes": mem_gpu32, "kernels": kernel_avgs(r32),
                      "series_form": r32["tuned"]},
        "batched": batched,
        "adjoint": adjoint,
        "pcg": pcg,
        "large": large,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def pcg_section(poba, torch, stream, results):
    """The comparison solvers on the benchmark workload (FP64 and FP32-bulk handles at their
    current linearisation, lambda = 1e-4): PCG on the reduced camera system with the
    Schur-Jacobi preconditioner and with the order-2 power series (PoCG), to relative residuals
    1e-2 and 1e-4, against the power-series solve (20 terms).  Times are CUDA events around one
    solve (median of 3); PCG synchronises once per iteration."""
    out = {}
    for name in ("fp64", "fp32_bulk"):
        h = results[name]["h"]
        poba.ba_linearize(h, want_cost=False)
        rows = []
        for precond, m in (("jacobi", 0), ("power", 2)):
            for rtol in (1e-2, 1e-4):
                ms, it = [], 0
                for _ in range(3):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    info = poba.ba_solve_schur_pcg(h, 1e-4, precond, m, rtol=rtol, max_iter=500)
                    b.record(stream)
                    stream.synchronize()
                    ms.append(a.elapsed_time(b))
                    it = info["iterations"]
                rows.append({"precond": precond, "m": m, "rtol": rtol, "iterations": it,
                             "ms": float(np.median(ms))})
        ms = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            info = poba.ba_solve_schur_power(h, 1e-4)
            b.record(stream)
            stream.synchronize()
            ms.append(a.elapsed_time(b))
        out[name] = {"pcg": rows, "power_series": {"terms": info["inner_iters"],
                                                    "ms": float(np.median(ms))}}
    out["config"] = {"workload": WORKLOAD, "lambda": 1e-4, "max_iter": 500}
    return out


def adjoint_section(args, poba, torch, stream, dev):
    """Differentiable BA: 200 cameras, 20,000 landmarks (about 80,000 observations), weights
    U(0.5, 1.5), FP64.  Forward: LM from x0 to func_tol (or 50 iterations).  Backward: the
    implicit-differentiation adjoint (damp, invert, the series with the default eps 0.01 and at
    most 20 terms, back-substitution, per-observation gradients) at the LM's final lambda, for a
    random dL/dx, with device inputs and outputs.  Both timed with CUDA events; the backward is
    repeated and the median reported."""
    p = bal_synth.preset("weighted_200c_20000l")
    to = lambda a: torch.as_tensor(a).to(dev)
    with torch.cuda.stream(stream):
        h = poba.ba_create(to(p.cams0), to(p.lms0), to(p.obs), to(p.cam_idx), to(p.lm_idx),
                           to(p.weights), options=poba.ba_default_options(), stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        steps = poba.ba_lm_solve(h)
        e1.record(stream)
        stream.synchronize()
        fwd_ms = e0.elapsed_time(e1)
        lam = poba.ba_get_lm_state(h)["lam"]
        rng = np.random.default_rng(0)
        g_c = to(rng.normal(size=(p.n_cams, 9)))
        g_l = to(rng.normal(size=(p.n_lms, 3)))
        d_obs = torch.empty((p.n_obs, 2), dtype=torch.float64, device=dev)
        d_w = torch.empty(p.n_obs, dtype=torch.float64, device=dev)
        for _ in range(3):
            poba.ba_adjoint(h, lam, g_c, g_l, d_obs, d_w)
        ms = []
        info = None
        for _ in range(20):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, info = poba.ba_adjoint(h, lam, g_c, g_l, d_obs, d_w)
            b.record(stream)
            stream.synchronize()
            ms.append(a.elapsed_time(b))
    bwd = float(np.median(ms))
    return {"metric": "adjoint backward passes/s (implicit differentiation, FP64)",
            "value": 1e3 / bwd, "unit": "backward/s", "backward_ms": bwd,
            "forward_ms": fwd_ms, "forward_lm_iterations": len(steps),
            "adjoint_lambda": lam, "adjoint_terms": info["inner_iters"],
            "config": {"workload": "weighted_200c_20000l", "n_cams": p.n_cams,
                       "n_lms": p.n_lms, "n_obs": p.n_obs, "weights": "U(0.5, 1.5)"}}


LARGE_WORKLOAD = "powerlaw_10000c_1000000l"


def large_section(args, poba, torch, stream, dev, max_over_ranks, barrier):
    """The large single problem (10,000 cameras, 1,000,000 landmarks, about 5.0M observations,
    power-law tracks on [2, 50]) in FP32 bulk: LM iterations/s from x0, series solves/s, the
    series term against the HBM roofline (its Jacobians, 0.48 GB, are well beyond L2, so no
    flush is needed) and the memory footprint next to an explicit block-sparse S."""
    p = bal_synth.preset(LARGE_WORKLOAD)
    to_dev = lambda a: torch.as_tensor(a).to(dev)
    cams0_d, lms0_d = to_dev(p.cams0), to_dev(p.lms0)
    with torch.cuda.stream(stream):
        h = poba.ba_create(cams0_d, lms0_d, to_dev(p.obs), to_dev(p.cam_idx), to_dev(p.lm_idx),
                           precision=poba.BA_FP32_BULK, stream=stream)
    tuned = poba.ba_autotune(h, trials=2)
    n_steps = max(3, min(args.steps, 20))

    def lm_steps(n):
        poba.ba_set_params(h, cams0_d, lms0_d)
        poba.ba_set_lm_state(h, 1e-4, 2.0, 0)
        evs = []
        with torch.cuda.stream(stream):
            for _ in range(n):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                poba.ba_lm_step(h)
                e1.record(stream)
                evs.append((e0, e1))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    lm_steps(max(3, args.warmup))
    poba.ba_set_timing(h, True)
    launches0 = poba.ba_kernel_launches(h)
    barrier()
    ms = lm_steps(n_steps)
    barrier()
    launches = poba.ba_kernel_launches(h) - launches0
    timing = poba.ba_get_timing(h)
    poba.ba_set_timing(h, False)
    total_ms = max_over_ranks(sum(ms))
    poba.ba_linearize(h, want_cost=False)
    evs = []
    n_solves = 10
    with torch.cuda.stream(stream):
        for _ in range(n_solves):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = poba.ba_solve_schur_power(h, 1e-4)
            e1.record(stream)
            evs.append((e0, e1))
    stream.synchronize()
    solve_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs))
    ms_t, cnt = timing["series_tile"]
    ms_c, _ = timing["series_camera"]
    avg_s = (ms_t + ms_c) / 1e3 / max(cnt, 1)
    nb, nf = series_term_units(p, 4)
    sched = poba.ba_get_schedule(h)
    nd = series_term_design_bytes(p, sched["n_group_slots"], 4)
    hbm_peak, hbm_kind, _, _ = measured_peaks()
    ach = nb / avg_s / 1e9
    out = {
        "metric": "LM iterations/s (large single problem, FP32 bulk)",
        "value": n_steps / (total_ms / 1e3),
        "unit": "LM iterations/s",
        "ms_per_step": total_ms / n_steps,
        "solves_per_s": n_solves / (solve_ms / 1e3),
        "solve_inner_iters": info["inner_iters"],
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ach / hbm_peak,
                     "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)"
                     if hbm_kind == "measured" else "fallback 6800 GB/s",
                     "kernel": "series term (tile phase, camera phase, two grid barriers)",
                     "series_form": tuned, "schedule": sched,
                     "algorithmic_bytes_per_term": nb,
                     "algorithmic_flops_per_term": nf, "design_bytes_per_term": nd,
                     "design_gbs": nd / avg_s / 1e9, "avg_term_us": avg_s * 1e6, "terms": cnt,
                     "achieved_tflops": nf / avg_s / 1e12,
                     "traffic": profiled_traffic("fp32_bulk", tuned["exec"], LARGE_WORKLOAD)},
        "kernels": {k: {"avg_us": (v[0] * 1e3 / v[1]) if v[1] else None, "count": v[1]}
                    for k, v in timing.items()},
        "gpu_launches": int(launches),
        "memory_bytes": poba.ba_memory_footprint(h),
        "explicit_S_bytes": explicit_s_bytes(p),
        "config": {"workload": LARGE_WORKLOAD, "n_cams": p.n_cams, "n_lms": p.n_lms,
                   "n_obs": p.n_obs, "tracks": "power law k^-2.14 on [2, 50], window max(2k, 64)",
                   "series": {"eps": 0.01, "max_inner": 20}, "lm": {"lambda0": 1e-4},
                   "steps": n_steps, "l2": "inputs larger than L2 (no flush)"},
    }
    poba.ba_destroy(h)
    return out


def batched_section(args, poba, torch, stream, dev, max_over_ranks, barrier):
    """Batched independent sub-problems (the PoST cluster solves): 256 problems of uneven sizes
    (cameras U{8..200}, landmarks U{500..20000}, tracks U{2..8}) in one batch handle, FP32 bulk,
    every kernel and the persistent series launch covering all problems.  A solve runs LM from
    x0 until every problem has met func_tol (each is frozen when it does) or 50 steps.  Per
    problem, its solve time is the device time from the start of the batch solve to the end of
    the step in which it converged.  The batch's Jacobians (about 1.2 GB) exceed the L2 cache,
    so no flush is needed between steps."""
    probs = bal_synth.make_batch(256)
    P = len(probs)
    hb = poba.batch_from_problems(probs, precision=poba.BA_FP32_BULK, stream=stream)
    cams0 = torch.as_tensor(np.concatenate([q.cams0 for q in probs])).to(dev)
    lms0 = torch.as_tensor(np.concatenate([q.lms0 for q in probs])).to(dev)

    def solve():
        poba.ba_set_params(hb, cams0, lms0)
        poba.ba_set_lm_state(hb, 1e-4, 2.0, 0)
        evs, done_at = [], [None] * P
        n_not_spd = 0
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(50):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                infos, active = poba.ba_lm_step_batch(hb)
                e1.record(stream)
                evs.append((e0, e1))
                for i, st in enumerate(infos):
                    if done_at[i] is None:
                        n_not_spd += int(st["not_spd"])
                        if st["converged"]:
                            done_at[i] = k
                if active == 0:
                    break
        stream.synchronize()
        wall = time.perf_counter() - t0
        cum = np.cumsum([a.elapsed_time(b) for a, b in evs])
        per = [cum[d] if d is not None else cum[-1] for d in done_at]
        return (float(cum[-1]), wall, per, len(evs), sum(d is not None for d in done_at),
                n_not_spd)

    solve()  # warm-up solve
    tuned = poba.ba_autotune(hb, trials=2)  # picks the series schedule and form (untimed)
    schedule = poba.ba_get_schedule(hb)
    solve()  # captures the LM-step graph for the tuned schedule (untimed)
    graph = poba.ba_get_step_graph(hb)
    launches0 = poba.ba_kernel_launches(hb)
    barrier()
    runs = [solve() for _ in range(max(1, args.batch_solves))]
    barrier()
    launches = poba.ba_kernel_launches(hb) - launches0
    dev_ms = max_over_ranks(sum(r[0] for r in runs))
    wall_s = max_over_ranks(sum(r[1] for r in runs))
    per = np.array(runs[-1][2])
    n_solves = len(runs)
    f32_costs = poba.ba_cost_batch(hb)
    # the plain FP64 path on the same batch: one solve, its time and the final costs
    del hb
    h64 = poba.batch_from_problems(probs, precision=poba.BA_FP64, stream=stream)
    poba.ba_autotune(h64, trials=1)
    poba.ba_set_params(h64, cams0, lms0)
    poba.ba_set_lm_state(h64, 1e-4, 2.0, 0)
    hb = h64
    r64 = solve()
    f64_costs = poba.ba_cost_batch(h64)
    ratio = f32_costs / f64_costs - 1.0
    return {
        "metric": "problems/s (batched sub-problems solved to func_tol, FP32 bulk)",
        "value": P * n_solves / (dev_ms / 1e3),
        "unit": "problems/s",
        "wall_value": P * n_solves / wall_s,
        "p50_solve_ms": float(np.percentile(per, 50)),
        "p99_solve_ms": float(np.percentile(per, 99)),
        "batch_solve_ms": dev_ms / n_solves,
        "lm_steps_per_solve": runs[-1][3],
        "converged": runs[-1][4],
        "not_spd_iterations": runs[-1][5],
        "series_form": tuned,
        "schedule": schedule,
        "step_graph": {"enabled": graph["enabled"], "kernels_per_step": graph["kernels_per_step"],
                       "host_calls_per_step": ("one cudaGraphLaunch (the whole LM step: "
                                               "linearisation gated on the device, series, "
                                               "decision, record copies) + one stream sync"
                                               if graph["enabled"] else "eager launches")},
        "fp64_batch": {"problems_per_s": P / (r64[0] / 1e3), "batch_solve_ms": r64[0],
                       "p50_solve_ms": float(np.percentile(r64[2], 50)),
                       "p99_solve_ms": float(np.percentile(r64[2], 99)),
                       "converged": r64[4], "lm_steps_per_solve": r64[3]},
        "final_cost_fp32_vs_fp64": {"median_rel": float(np.median(ratio)),
                                    "max_abs_rel": float(np.abs(ratio).max())},
        "gpu_launches": int(launches),
        "solves": n_solves,
        "memory_bytes": poba.ba_memory_footprint(hb),
        "config": {"workload": "batch_256_uneven", "n_problems": P,
                   "n_cams": int(sum(q.n_cams for q in probs)),
                   "n_lms": int(sum(q.n_lms for q in probs)),
                   "n_obs": int(sum(q.n_obs for q in probs)),
                   "sizes": "cameras U{8..200}, landmarks U{500..20000}, tracks U{2..8}",
                   "lm": {"lambda0": 1e-4, "func_tol": 1e-6, "max_lm": 50},
                   "l2": "inputs larger than L2 (no flush)"},
    }


def schedule_slots(p, tile_obs=256, tile_lms=256, tile_cams=128) -> int:
    """Number of (tile, camera) slots of the library's schedule: landmarks ordered by their
    smallest observing camera, packed greedily into tiles of whole tracks (at most tile_obs
    observations, tile_lms landmarks, tile_cams distinct cameras)."""
    key = np.full(p.n_lms, p.n_cams, dtype=np.int64)
    np.minimum.at(key, p.lm_idx, p.cam_idx)
    lm_order = np.argsort(key, kind="stable")
    rank = np.empty_like(lm_order)
    rank[lm_order] = np.arange(p.n_lms)
    order = np.lexsort((p.cam_idx, rank[p.lm_idx]))
    cams = p.cam_idx[order].tolist()
    seg = np.concatenate([[0], np.cumsum(np.bincount(rank[p.lm_idx], minlength=p.n_lms))]).tolist()
    stamp = [-1] * p.n_cams
    tile = obs = lms = ncam = slots = 0
    for i in range(p.n_lms):
        a, b = seg[i], seg[i + 1]
        fresh = sum(1 for c in cams[a:b] if stamp[c] != tile)
        if lms > 0 and (obs + b - a > tile_obs or lms + 1 > tile_lms or ncam + fresh > tile_cams):
            slots += ncam
            tile += 1
            obs = lms = ncam = 0
            fresh = b - a
        for c in cams[a:b]:
            stamp[c] = tile
        obs += b - a
        lms += 1
        ncam += fresh
    return slots + ncam


# ---------------------------------------------------------------------------------------
ORACLE_ENV_1T = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def run_oracle_workers(args, solver: str, seconds: float, n: int) -> list[dict]:
    """Run n oracle LM workers (each single-threaded, in its own process) on the workload for
    about `seconds` each, started together, and return their reports."""
    env = dict(os.environ)
    for k in ORACLE_ENV_1T:
        env[k] = "1"
    with tempfile.TemporaryDirectory(prefix="poba_oracle_") as sync:
        cmd = [sys.executable, os.path.abspath(__file__), "--cpu-baseline-worker", "--workload",
               args.workload, "--cpu-seconds", str(seconds), "--cpu-solver", solver,
               "--cpu-sync-dir", sync, "--cpu-sync-n", str(n)]
        procs = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                  text=True) for _ in range(n)]
        reports = []
        try:
            for pr in procs:
                out, err = pr.communicate(timeout=600 + 4 * seconds)
                if pr.returncode != 0:
                    raise RuntimeError(f"oracle worker exited {pr.returncode}: {err[-300:]}")
                reports.append(json.loads(out.strip().splitlines()[-1]))
        finally:
            for pr in procs:
                if pr.poll() is None:
                    pr.kill()
                    pr.wait()
    return reports


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def host_free_bytes() -> int | None:
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError, AttributeError):
        return None


def cpu_baseline(args) -> dict:
    """The FP64 oracle (as it stands) on the host cores, on the same workload:
      * the reported value: single-threaded LM iterations with the power-series solve
        (BLAS / OpenMP threads pinned to 1, in a subprocess), with its peak RSS;
      * `direct`: the same LM with the oracle's exact solve of the reduced system (explicit
        block-sparse S, Schur-Jacobi PCG to 1e-12), single-threaded;
      * `all_cores`: independent single-threaded power-series LM replicas, one per host core
        (capped so their resident sets fit in half the free host memory), started together;
        value = all replicas' iterations / the span from the first start to the last end."""
    unit = "LM iterations/s"
    try:
        (d,) = run_oracle_workers(args, "power", args.cpu_seconds, 1)
    except Exception as e:  # report, do not hide
        return {"value": None, "unit": unit, "cores": 1, "kind": "oracle",
                "sample": f"failed: {e}"}
    line = {"value": d["iters"] / d["seconds"], "unit": unit, "cores": 1, "kind": "oracle",
            "sample": f"{d['iters']} oracle LM iterations from x0 on the full {args.workload} "
                      f"problem ({d['seconds']:.1f} s; numpy/scipy, 1 thread)",
            "peak_rss_bytes": d["peak_rss_bytes"]}
    side = max(args.cpu_seconds / 2, 0.1)
    try:
        (e,) = run_oracle_workers(args, "direct", side, 1)
        line["direct"] = {
            "value": e["iters"] / e["seconds"], "unit": unit, "cores": 1,
            "solver": "explicit block-sparse S, Schur-Jacobi PCG to 1e-12",
            "sample": f"{e['iters']} oracle LM iterations from x0 ({e['seconds']:.1f} s)",
            "peak_rss_bytes": e["peak_rss_bytes"]}
    except Exception as ex:
        line["direct"] = {"value": None, "unit": unit, "sample": f"failed: {ex}"}
    cores = host_cores()
    free = host_free_bytes()
    n = cores
    if free is not None:
        n = max(1, min(cores, int(0.5 * free // max(d["peak_rss_bytes"], 1))))
    try:
        reps = run_oracle_workers(args, "power", side, n)
        span = max(r["end"] for r in reps) - min(r["start"] for r in reps)
        iters = sum(r["iters"] for r in reps)
        line["all_cores"] = {
            "value": iters / span, "unit": unit, "cores": n, "host_cores": cores,
            "sample": f"{n} independent single-threaded oracle LM replicas, {iters} iterations "
                      f"in {span:.1f} s",
            "peak_rss_bytes_per_replica": max(r["peak_rss_bytes"] for r in reps)}
    except Exception as ex:
        line["all_cores"] = {"value": None, "unit": unit, "sample": f"failed: {ex}"}
    return line


def oracle_lm_iterations(p, n: int, solver: str = "power") -> int:
    """n LM iterations of the oracle's own loop (oracle.lm.lm_solve) from x0, restarting from x0
    after convergence or 50 iterations, as the library arm does.  Within a solve the
    linearisation is kept across rejected steps (lm_solve rebuilds it only after an accepted
    one).  Returns the iterations run (n)."""
    from oracle import lm as olm
    done = 0
    while done < n:
        _, _, hist = olm.lm_solve(p, olm.Options(max_lm=min(50, n - done)), solver=solver)
        done += len(hist)
    return done


def cpu_baseline_worker(args):
    import resource
    p = bal_synth.preset(args.workload)
    if args.cpu_sync_dir:
        # start together: announce readiness, then wait (bounded) for the others
        open(os.path.join(args.cpu_sync_dir, f"ready.{os.getpid()}"), "w").close()
        t_wait = time.monotonic()
        while (len(os.listdir(args.cpu_sync_dir)) < args.cpu_sync_n
               and time.monotonic() - t_wait < 300):
            time.sleep(0.01)
    start = time.time()
    t0 = time.perf_counter()
    # one iteration sizes the sample, then as many more as fit the time budget (a new solve
    # from x0; each solve keeps its linearisation across rejected steps)
    n = oracle_lm_iterations(p, 1, args.cpu_solver)
    t1 = time.perf_counter() - t0
    more = int(max(0.0, args.cpu_seconds - t1) // max(t1, 1e-9))
    if more:
        n += oracle_lm_iterations(p, more, args.cpu_solver)
    seconds = time.perf_counter() - t0
    rss = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss * 1024  # KiB on Linux
    print(json.dumps({"iters": n, "seconds": seconds, "start": start, "end": start + seconds,
                      "peak_rss_bytes": rss}))


def run_reference(args):
    """Reference arm: the FP64 CPU oracle's LM loop timed on the host cores (the paper ships no
    code): W untimed warm-up iterations, then K timed ones (fewer only if K iterations would
    exceed REFERENCE_BUDGET_S at the warm-up's pace; the line says so), on the same workload and
    with the same config as the library arm."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    p = bal_synth.preset(args.workload)
    warm = max(0, args.warmup)
    tw = time.perf_counter()
    if warm:
        oracle_lm_iterations(p, warm)
    per = (time.perf_counter() - tw) / warm if warm else None
    steps = max(1, args.steps)
    if per and per * steps > REFERENCE_BUDGET_S:
        steps = max(1, int(REFERENCE_BUDGET_S // per))
    t0 = time.perf_counter()
    n = oracle_lm_iterations(p, steps)
    dt = time.perf_counter() - t0
    v = n / dt
    capped = "" if n == args.steps else f" (of {args.steps} requested: {REFERENCE_BUDGET_S:.0f} s cap)"
    sample = (f"{n} oracle LM iterations{capped} after {warm} warm-up iterations, on the full "
              f"{args.workload} problem from x0 (oracle.lm.lm_solve: linearisation kept across "
              f"rejected steps, restart after convergence or 50 iterations), numpy/scipy FP64, "
              f"1 thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "LM iterations/s",
        "n_gpus": world, "steps": n, "warmup": warm, "ms_per_step": 1e3 * dt / n,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": data_note(args.workload),
        "config": headline_config(args.workload, p, world),
        "cpu_baseline": {"value": v, "unit": "LM iterations/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "LM iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_fp64_probe(args):
    """The FP64 FMA rate of the device (ba_probe_fp64_fma, 5 launches of each residency) with
    the SM clocks sampled while it runs: per launch TFLOP/s and the FMA/clk/SM it implies at the
    median sampled clock."""
    import torch
    import paper_2204_12834_gb300 as poba
    from paper_2204_12834_gb300 import build as pbuild
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pbuild.build()
    poba.library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = ClockSampler(local)
    clocks.start()
    rows = []
    for bps in (1, 2, 4, 8):
        for _ in range(5):
            r = poba.ba_probe_fp64_fma(bps, 1 << 16, stream)
            rows.append({"blocks_per_sm": bps, "tflops": r["flops_per_s"] / 1e12, "ms": r["ms"]})
    clk = clocks.stop()
    mhz = clk.get("sm_mhz") or DEFAULT_MAX_SM_MHZ
    best = max(rows, key=lambda d: d["tflops"])
    print(json.dumps({
        "probe": "ba_probe_fp64_fma", "sms": sms, "threads_per_block": 256, "fma_chains": 8,
        "iters": 1 << 16, "launches": rows, "best_tflops": best["tflops"],
        "fma_per_clk_per_sm_at_median_clock": best["tflops"] * 1e12 / (2 * sms * mhz * 1e6),
        "derived_peak_tflops": fp64_peak_tflops(sms, clk.get("sm_max_mhz")), "clocks": clk}),
        flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_baseline_worker:
        return cpu_baseline_worker(args)
    if args.fp64_probe:
        return run_fp64_probe(args)
    if args.impl == "reference":
        if os.environ.get("POBA_REFERENCE_CHILD") != "1":
            # pin BLAS / OpenMP to one thread so the reported core count is exact
            env = dict(os.environ, POBA_REFERENCE_CHILD="1", OMP_NUM_THREADS="1",
                       OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
            os.execve(sys.executable, [sys.executable, os.path.abspath(__file__)] + sys.argv[1:], env)
        return run_reference(args)
    return run_poba(args)


if __name__ == "__main__":
    main()
