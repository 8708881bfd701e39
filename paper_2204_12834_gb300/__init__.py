"""GB300-native Power Bundle Adjustment (Weber et al., "Power Bundle Adjustment for
Large-Scale 3D Reconstruction").

Python binding of libpoba (include/poba.h).  Each ``ba_*`` function here marshals arguments to
the C entry point of the same name; every step of the solve runs in the library's CUDA kernels
(no CPU fallback: the import of the binding fails when libpoba.so is missing).

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA memory); outputs are
returned as numpy arrays unless a torch CUDA tensor is passed to fill.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import _lib
from ._lib import BA_FP64, BA_FP32_BULK, Options, ProblemDesc, SeriesInfo, StepInfo

__all__ = ["PobaError", "Handle", "ba_default_options", "ba_create", "ba_set_options",
           "ba_linearize", "ba_solve_schur_power", "ba_lm_step", "ba_lm_solve", "ba_cost",
           "ba_get_params", "ba_set_params", "ba_get_step", "ba_get_linearization",
           "ba_get_blocks", "ba_get_lm_state", "ba_set_lm_state", "ba_memory_footprint",
           "ba_kernel_launches", "ba_set_timing", "ba_get_timing", "ba_destroy", "BA_FP64",
           "BA_FP32_BULK", "library", "from_problem", "ba_cost_noalloc", "BA_NOALLOC_MAX_CAMS",
           "ba_get_series_trace", "ba_set_barrier_timeout", "ba_create_batch",
           "ba_get_batch_layout", "ba_get_series_state", "ba_lm_step_batch", "ba_lm_solve_batch",
           "ba_cost_batch", "batch_from_problems", "ba_autotune", "ba_adjoint",
           "ba_solve_schur_pcg", "ba_get_schedule", "ba_set_schedule", "ba_set_step_graph",
           "ba_get_step_graph", "ba_probe_fp64_fma", "ba_debug_checks"]

BA_NOALLOC_MAX_CAMS = 4096


class PobaError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        self.status_name = _lib.STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.status_name}: {message}")


def library() -> C.CDLL:
    return _lib.load()


def _check(status: int, where: str):
    if status != _lib.BA_OK:
        msg = library().ba_last_error().decode(errors="replace")
        raise PobaError(status, where, msg)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype):
    """(pointer, ptr_kind, keepalive) for a numpy array or torch tensor of the given dtype."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            a = a.to(tdt).contiguous()
        return a.data_ptr(), (1 if a.is_cuda else 0), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr


@dataclass
class Handle:
    ptr: C.c_void_p
    n_cams: int
    n_lms: int
    n_obs: int
    precision: int
    n_problems: int = 1

    def __del__(self):
        try:
            if self.ptr:
                library().ba_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def ba_default_options(**overrides) -> Options:
    o = Options()
    _check(library().ba_default_options(C.byref(o)), "ba_default_options")
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _fill_desc(d: ProblemDesc, cams, lms, obs, cam_idx, lm_idx, weights, precision, stream, keep):
    n_c = int(cams.shape[0])
    n_l = int(lms.shape[0])
    n_o = int(obs.shape[0])
    kinds = set()
    d.n_cams, d.n_lms, d.n_obs = n_c, n_l, n_o
    for field, arr, dt in (("cams", cams, np.float64), ("lms", lms, np.float64),
                           ("obs", obs, np.float64), ("cam_idx", cam_idx, np.int32),
                           ("lm_idx", lm_idx, np.int32), ("weights", weights, np.float64)):
        p, kind, k = _ptr(arr, dt)
        setattr(d, field, p)
        keep.append(k)
        if kind is not None:
            kinds.add(kind)
    if len(kinds) > 1:
        raise ValueError("all inputs must live in the same memory (all host or all device)")
    d.ptr_kind = kinds.pop() if kinds else 0
    d.precision = int(precision)
    if stream is not None:
        d.cuda_stream = int(getattr(stream, "cuda_stream", stream)) or None
    return n_c, n_l, n_o


def ba_create(cams, lms, obs, cam_idx, lm_idx, weights=None, precision: int = BA_FP64,
              options: Optional[Options] = None, stream=None) -> Handle:
    """Create a problem handle (copies every input)."""
    keep = []
    d = ProblemDesc()
    n_c, n_l, n_o = _fill_desc(d, cams, lms, obs, cam_idx, lm_idx, weights, precision, stream, keep)
    out = C.c_void_p()
    opts = options if options is not None else ba_default_options()
    _check(library().ba_create(C.byref(d), C.byref(opts), C.byref(out)), "ba_create")
    return Handle(out, n_c, n_l, n_o, int(precision))


def ba_create_batch(problems, precision: int = BA_FP64, options: Optional[Options] = None,
                    stream=None) -> Handle:
    """Create a batch handle from a sequence of (cams, lms, obs, cam_idx, lm_idx, weights)
    tuples, indices local to each problem.  The handle's arrays are the problems'
    concatenated in order (offsets: ba_get_batch_layout)."""
    keep = []
    descs = (ProblemDesc * len(problems))()
    tot = [0, 0, 0]
    for i, pr in enumerate(problems):
        cams, lms, obs, ci, li = pr[:5]
        w = pr[5] if len(pr) > 5 else None
        sizes = _fill_desc(descs[i], cams, lms, obs, ci, li, w, precision,
                           stream if i == 0 else None, keep)
        tot = [a + b for a, b in zip(tot, sizes)]
    out = C.c_void_p()
    opts = options if options is not None else ba_default_options()
    _check(library().ba_create_batch(descs, len(problems), C.byref(opts), C.byref(out)),
           "ba_create_batch")
    return Handle(out, tot[0], tot[1], tot[2], int(precision), len(problems))


def batch_from_problems(problems, precision: int = BA_FP64, options: Optional[Options] = None,
                        stream=None) -> Handle:
    """ba_create_batch from bal_synth.Problem-like objects."""
    return ba_create_batch([(p.cams0, p.lms0, p.obs, p.cam_idx, p.lm_idx, p.weights)
                            for p in problems], precision=precision, options=options,
                           stream=stream)


def ba_get_batch_layout(h: Handle):
    """(cam_off, lm_off), each [P + 1]: problem p owns cameras cam_off[p]:cam_off[p+1] and
    landmarks lm_off[p]:lm_off[p+1] of the handle's arrays."""
    n = C.c_int32()
    _check(library().ba_get_batch_layout(h.ptr, C.byref(n), None, None), "ba_get_batch_layout")
    co = np.empty(n.value + 1, dtype=np.int32)
    lo = np.empty(n.value + 1, dtype=np.int32)
    _check(library().ba_get_batch_layout(h.ptr, C.byref(n), co.ctypes.data, lo.ctypes.data),
           "ba_get_batch_layout")
    return co, lo


def _series_dict(info: SeriesInfo) -> dict:
    return dict(inner_iters=info.inner_iters, stopped=info.stopped, stop_value=info.stop_value,
                x_norm=info.x_norm, lam=info.lambda_)


def ba_get_series_state(h: Handle) -> list:
    infos = (SeriesInfo * h.n_problems)()
    _check(library().ba_get_series_state(h.ptr, infos), "ba_get_series_state")
    return [_series_dict(infos[i]) for i in range(h.n_problems)]


def ba_lm_step_batch(h: Handle):
    """(list of per-problem step dicts, number of problems still active)."""
    infos = (StepInfo * h.n_problems)()
    n = C.c_int32()
    _check(library().ba_lm_step_batch(h.ptr, infos, C.byref(n)), "ba_lm_step_batch")
    return [_step_dict(infos[i]) for i in range(h.n_problems)], n.value


def ba_lm_solve_batch(h: Handle):
    """(list of each problem's last step dict, number of batch steps run)."""
    infos = (StepInfo * h.n_problems)()
    n = C.c_int32()
    _check(library().ba_lm_solve_batch(h.ptr, infos, C.byref(n)), "ba_lm_solve_batch")
    return [_step_dict(infos[i]) for i in range(h.n_problems)], n.value


def ba_cost_batch(h: Handle) -> np.ndarray:
    c = np.empty(h.n_problems, dtype=np.float64)
    _check(library().ba_cost_batch(h.ptr, c.ctypes.data), "ba_cost_batch")
    return c


def ba_set_options(h: Handle, options: Options):
    _check(library().ba_set_options(h.ptr, C.byref(options)), "ba_set_options")


def ba_linearize(h: Handle, want_cost: bool = True):
    c = C.c_double()
    _check(library().ba_linearize(h.ptr, C.byref(c) if want_cost else None), "ba_linearize")
    return c.value if want_cost else None


def ba_solve_schur_power(h: Handle, lam: float, want_info: bool = True):
    info = SeriesInfo()
    _check(library().ba_solve_schur_power(h.ptr, float(lam), C.byref(info) if want_info else None),
           "ba_solve_schur_power")
    if not want_info:
        return None
    return _series_dict(info)


def _step_dict(s: StepInfo) -> dict:
    return dict(cost_before=s.cost_before, cost_after=s.cost_after, lam=s.lambda_,
                gain_ratio=s.gain_ratio, model_decrease=s.model_decrease, stop_value=s.stop_value,
                accepted=bool(s.accepted), inner=s.inner_iters, converged=bool(s.converged),
                it=s.iteration, not_spd=bool(s.not_spd))


def ba_lm_step(h: Handle) -> dict:
    s = StepInfo()
    _check(library().ba_lm_step(h.ptr, C.byref(s)), "ba_lm_step")
    return _step_dict(s)


def ba_lm_solve(h: Handle, max_lm: int = 50) -> list:
    trace = (StepInfo * max(1, max_lm))()
    n = C.c_int32()
    _check(library().ba_lm_solve(h.ptr, trace, C.byref(n)), "ba_lm_solve")
    return [_step_dict(trace[i]) for i in range(n.value)]


def ba_cost(h: Handle) -> float:
    c = C.c_double()
    _check(library().ba_cost(h.ptr, C.byref(c)), "ba_cost")
    return c.value


def _out(shape, dst):
    if dst is None:
        a = np.empty(shape, dtype=np.float64)
        return a, a.ctypes.data, 0
    if _is_torch(dst):
        return dst, dst.data_ptr(), (1 if dst.is_cuda else 0)
    return dst, dst.ctypes.data, 0


def ba_get_params(h: Handle, cams_out=None, lms_out=None):
    c, cp, k1 = _out((h.n_cams, 9), cams_out)
    l, lp, k2 = _out((h.n_lms, 3), lms_out)
    if k1 != k2:
        raise ValueError("outputs must live in the same memory")
    _check(library().ba_get_params(h.ptr, cp, lp, k1), "ba_get_params")
    return c, l


def ba_set_params(h: Handle, cams, lms):
    cp, k1, kc = _ptr(cams, np.float64)
    lp, k2, kl = _ptr(lms, np.float64)
    kind = k1 if k1 is not None else (k2 if k2 is not None else 0)
    _check(library().ba_set_params(h.ptr, cp, lp, kind), "ba_set_params")


def ba_get_step(h: Handle, dx_p_out=None, dx_l_out=None):
    a, ap, k1 = _out((h.n_cams, 9), dx_p_out)
    b, bp, k2 = _out((h.n_lms, 3), dx_l_out)
    if k1 != k2:
        raise ValueError("outputs must live in the same memory")
    _check(library().ba_get_step(h.ptr, ap, bp, k1), "ba_get_step")
    return a, b


def ba_get_linearization(h: Handle):
    r = np.empty((h.n_obs, 2))
    Jp = np.empty((h.n_obs, 2, 9))
    Jl = np.empty((h.n_obs, 2, 3))
    _check(library().ba_get_linearization(h.ptr, r.ctypes.data, Jp.ctypes.data, Jl.ctypes.data, 0),
           "ba_get_linearization")
    return r, Jp, Jl


def ba_get_blocks(h: Handle):
    U = np.empty((h.n_cams, 9, 9))
    V = np.empty((h.n_lms, 3, 3))
    bp = np.empty(h.n_cams * 9)
    bl = np.empty(h.n_lms * 3)
    _check(library().ba_get_blocks(h.ptr, U.ctypes.data, V.ctypes.data, bp.ctypes.data,
                                   bl.ctypes.data, 0), "ba_get_blocks")
    return U, V, bp, bl


def ba_get_lm_state(h: Handle) -> dict:
    lam, nu, cost = C.c_double(), C.c_double(), C.c_double()
    it = C.c_int32()
    _check(library().ba_get_lm_state(h.ptr, C.byref(lam), C.byref(nu), C.byref(it), C.byref(cost)),
           "ba_get_lm_state")
    return dict(lam=lam.value, nu=nu.value, iteration=it.value, cost=cost.value)


def ba_set_lm_state(h: Handle, lam: float, nu: float, iteration: int):
    _check(library().ba_set_lm_state(h.ptr, float(lam), float(nu), int(iteration)), "ba_set_lm_state")


def ba_memory_footprint(h: Handle) -> int:
    b = C.c_uint64()
    _check(library().ba_memory_footprint(h.ptr, C.byref(b)), "ba_memory_footprint")
    return b.value


def ba_kernel_launches(h: Handle) -> int:
    b = C.c_uint64()
    _check(library().ba_kernel_launches(h.ptr, C.byref(b)), "ba_kernel_launches")
    return b.value


def ba_set_timing(h: Handle, enable: bool = True):
    _check(library().ba_set_timing(h.ptr, 1 if enable else 0), "ba_set_timing")


def ba_get_timing(h: Handle) -> dict:
    """{class: (total_ms, count)} for the kernel classes of include/poba.h."""
    t = _lib.Timing()
    _check(library().ba_get_timing(h.ptr, C.byref(t)), "ba_get_timing")
    return {name: (t.ms[i], int(t.count[i])) for i, name in enumerate(_lib.TIMING_CLASSES)}


def ba_cost_noalloc(cams, lms, obs, cam_idx, lm_idx, cost_out, weights=None, stream=None):
    """Allocation-free cost evaluation: every argument is a CUDA tensor on the current device
    (float64 / int32, contiguous) and the result is written to the one-element CUDA tensor
    cost_out.  Nothing is allocated and nothing is synchronised."""
    import torch
    args = []
    for a, dt in ((cams, torch.float64), (lms, torch.float64), (obs, torch.float64),
                  (cam_idx, torch.int32), (lm_idx, torch.int32), (weights, torch.float64),
                  (cost_out, torch.float64)):
        if a is None:
            args.append(None)
            continue
        if not (_is_torch(a) and a.is_cuda and a.is_contiguous() and a.dtype == dt):
            raise ValueError("ba_cost_noalloc takes contiguous CUDA tensors of dtype float64 "
                             "(indices int32); no conversion is made")
        args.append(a.data_ptr())
    st = None
    if stream is not None:
        st = int(getattr(stream, "cuda_stream", stream)) or None
    _check(library().ba_cost_noalloc(int(cams.shape[0]), int(lms.shape[0]), int(obs.shape[0]),
                                     *args, st), "ba_cost_noalloc")


def ba_debug_checks(h: Handle) -> dict:
    """The debug build's check record and buffer guards (see poba.h): {"enabled", "site",
    "count", "index"}; the record is cleared."""
    e, site, cnt, idx = C.c_int32(), C.c_uint32(), C.c_uint32(), C.c_int64()
    _check(library().ba_debug_checks(h.ptr, C.byref(e), C.byref(site), C.byref(cnt), C.byref(idx)),
           "ba_debug_checks")
    return {"enabled": bool(e.value), "site": site.value, "count": cnt.value, "index": idx.value}


def ba_probe_fp64_fma(blocks_per_sm: int = 4, iters: int = 1 << 16, stream=None) -> dict:
    """The device's FP64 FMA rate (see poba.h): {"flops_per_s", "ms"} of one timed launch."""
    st = None
    if stream is not None:
        st = int(getattr(stream, "cuda_stream", stream)) or None
    f, ms = C.c_double(), C.c_double()
    _check(library().ba_probe_fp64_fma(int(blocks_per_sm), int(iters), st, C.byref(f),
                                       C.byref(ms)), "ba_probe_fp64_fma")
    return {"flops_per_s": f.value, "ms": ms.value}


def ba_get_series_trace(h: Handle):
    """[terms, 5] ns timeline of block 0 in the last persistent series solve (see poba.h)."""
    buf = np.zeros(64 * 5, dtype=np.int64)
    n = C.c_int32()
    _check(library().ba_get_series_trace(h.ptr, buf.ctypes.data, buf.size, C.byref(n)),
           "ba_get_series_trace")
    return buf[: 5 * n.value].reshape(n.value, 5)


def ba_set_barrier_timeout(h: Handle, cycles: int):
    _check(library().ba_set_barrier_timeout(h.ptr, int(cycles)), "ba_set_barrier_timeout")


def ba_autotune(h: Handle, trials: int = 3) -> dict:
    """Time the series schedules (form, residency, group size) on the current linearisation and
    keep the fastest for series_exec 2.  Returns {"exec": 1 | 3 | 4, "blocks_per_sm": k}."""
    e, k = C.c_int32(), C.c_int32()
    _check(library().ba_autotune(h.ptr, int(trials), C.byref(e), C.byref(k)), "ba_autotune")
    return {"exec": e.value, "blocks_per_sm": k.value}


def ba_set_step_graph(h: Handle, enable: bool = True):
    """LM steps replay one captured CUDA graph (the default) or launch kernel by kernel."""
    _check(library().ba_set_step_graph(h.ptr, 1 if enable else 0), "ba_set_step_graph")


def ba_get_step_graph(h: Handle) -> dict:
    """{"enabled": bool, "kernels_per_step": int (0 before the first captured step)}."""
    e, k = C.c_int32(), C.c_int32()
    _check(library().ba_get_step_graph(h.ptr, C.byref(e), C.byref(k)), "ba_get_step_graph")
    return {"enabled": bool(e.value), "kernels_per_step": k.value}


def ba_get_schedule(h: Handle) -> dict:
    """The handle's series schedule: group_obs, tail_parts, series_exec, blocks_per_sm,
    n_groups, n_chunks, n_group_slots."""
    s = _lib.Schedule()
    _check(library().ba_get_schedule(h.ptr, C.byref(s)), "ba_get_schedule")
    return {name: getattr(s, name) for name, _ in _lib.Schedule._fields_}


def ba_set_schedule(h: Handle, group_obs: Optional[int] = None, series_exec: Optional[int] = None,
                    blocks_per_sm: Optional[int] = None, tail_parts: Optional[int] = None):
    """Change the series schedule; arguments left as None keep their current value."""
    cur = ba_get_schedule(h)
    s = _lib.Schedule()
    s.group_obs = int(cur["group_obs"] if group_obs is None else group_obs)
    s.tail_parts = int(cur["tail_parts"] if tail_parts is None else tail_parts)
    s.series_exec = int(cur["series_exec"] if series_exec is None else series_exec)
    s.blocks_per_sm = int(cur["blocks_per_sm"] if blocks_per_sm is None else blocks_per_sm)
    _check(library().ba_set_schedule(h.ptr, C.byref(s)), "ba_set_schedule")


def ba_adjoint(h: Handle, lam: float, g_cams, g_lms, d_obs=None, d_weights=None,
               want_weights: bool = True):
    """Implicit-differentiation adjoint at the current state (see include/poba.h): returns
    (d_obs [n_obs, 2], d_weights [n_obs] or None, series info).  g_cams / g_lms are numpy arrays
    or torch tensors; with CUDA tensors the outputs are CUDA tensors (pass d_obs / d_weights to
    fill preallocated ones)."""
    gp, k1, kg = _ptr(g_cams, np.float64)
    gl, k2, kl = _ptr(g_lms, np.float64)
    if k1 != k2:
        raise ValueError("g_cams and g_lms must live in the same memory")
    if k1 == 1:
        import torch
        dev = kg.device
        if d_obs is None:
            d_obs = torch.empty((h.n_obs, 2), dtype=torch.float64, device=dev)
        if d_weights is None and want_weights:
            d_weights = torch.empty(h.n_obs, dtype=torch.float64, device=dev)
        po, pw = d_obs.data_ptr(), (d_weights.data_ptr() if d_weights is not None else None)
    else:
        if d_obs is None:
            d_obs = np.empty((h.n_obs, 2))
        if d_weights is None and want_weights:
            d_weights = np.empty(h.n_obs)
        po, pw = d_obs.ctypes.data, (d_weights.ctypes.data if d_weights is not None else None)
    info = SeriesInfo()
    _check(library().ba_adjoint(h.ptr, float(lam), gp, gl, po, pw, k1, C.byref(info)),
           "ba_adjoint")
    return d_obs, d_weights, _series_dict(info)


def ba_solve_schur_pcg(h: Handle, lam: float, precond: str = "jacobi", m: int = 2,
                       rtol: float = 1e-10, max_iter: int = 500) -> dict:
    """PCG on the reduced camera system; precond "jacobi" (Schur-Jacobi) or "power" (order-m
    series, PoCG).  The step is read with ba_get_step."""
    info = _lib.PcgInfo()
    code = {"jacobi": 0, "power": 1}[precond]
    _check(library().ba_solve_schur_pcg(h.ptr, float(lam), code, int(m), float(rtol),
                                        int(max_iter), C.byref(info)), "ba_solve_schur_pcg")
    return dict(iterations=info.iterations, converged=bool(info.converged),
                rel_residual=info.rel_residual, lam=info.lambda_)


def ba_destroy(h: Handle):
    if h.ptr:
        _check(library().ba_destroy(h.ptr), "ba_destroy")
        h.ptr = None


def from_problem(problem, precision: int = BA_FP64, options: Optional[Options] = None,
                 stream=None) -> Handle:
    """ba_create from a bal_synth.Problem-like object (cams0, lms0, obs, indices, weights)."""
    return ba_create(problem.cams0, problem.lms0, problem.obs, problem.cam_idx, problem.lm_idx,
                     problem.weights, precision=precision, options=options, stream=stream)
