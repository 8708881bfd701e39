"""ctypes declarations for libpoba.so (mirrors include/poba.h)."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpoba.so")
CHECKS_LIB_PATH = os.path.join(_PKG, "libpoba_checks.so")

BA_OK = 0
STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_CUDA", 3: "BA_ERR_OOM",
                4: "BA_ERR_NOT_SPD", 5: "BA_ERR_NONFINITE", 6: "BA_ERR_NOT_LINEARIZED",
                7: "BA_ERR_TIMEOUT", 8: "BA_ERR_CHECK"}
BA_FP64 = 0
BA_FP32_BULK = 1


class ProblemDesc(C.Structure):
    _fields_ = [("n_cams", C.c_int32), ("n_lms", C.c_int32), ("n_obs", C.c_int32),
                ("cams", C.c_void_p), ("lms", C.c_void_p), ("obs", C.c_void_p),
                ("cam_idx", C.c_void_p), ("lm_idx", C.c_void_p), ("weights", C.c_void_p),
                ("ptr_kind", C.c_int32), ("precision", C.c_int32), ("cuda_stream", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("func_tol", C.c_double), ("eps", C.c_double),
                ("max_lm", C.c_int32), ("max_inner", C.c_int32), ("damping_mode", C.c_int32),
                ("series_exec", C.c_int32)]


class SeriesInfo(C.Structure):
    _fields_ = [("inner_iters", C.c_int32), ("stopped", C.c_int32), ("stop_value", C.c_double),
                ("x_norm", C.c_double), ("lambda_", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("cost_before", C.c_double), ("cost_after", C.c_double), ("lambda_", C.c_double),
                ("gain_ratio", C.c_double), ("model_decrease", C.c_double),
                ("stop_value", C.c_double), ("accepted", C.c_int32), ("inner_iters", C.c_int32),
                ("converged", C.c_int32), ("iteration", C.c_int32), ("not_spd", C.c_int32)]


class PcgInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32),
                ("rel_residual", C.c_double), ("lambda_", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("group_obs", C.c_int32), ("tail_parts", C.c_int32), ("series_exec", C.c_int32),
                ("blocks_per_sm", C.c_int32),
                ("n_groups", C.c_int32), ("n_chunks", C.c_int32), ("n_group_slots", C.c_int32)]


TIMING_CLASSES = ["linearize", "damp_invert", "rhs", "series_tile", "series_camera", "backsub",
                  "evaluate"]


class Timing(C.Structure):
    _fields_ = [("ms", C.c_double * 7), ("count", C.c_uint64 * 7)]


# name -> (restype, argtypes); every symbol declared in include/poba.h
SIGNATURES = {
    "ba_default_options": (C.c_int, [C.POINTER(Options)]),
    "ba_create": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(Options), C.POINTER(C.c_void_p)]),
    "ba_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "ba_linearize": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "ba_solve_schur_power": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(SeriesInfo)]),
    "ba_lm_step": (C.c_int, [C.c_void_p, C.POINTER(StepInfo)]),
    "ba_lm_solve": (C.c_int, [C.c_void_p, C.POINTER(StepInfo), C.POINTER(C.c_int32)]),
    "ba_cost": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "ba_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "ba_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "ba_get_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "ba_get_linearization": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "ba_get_blocks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "ba_get_lm_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "ba_set_lm_state": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int32]),
    "ba_memory_footprint": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "ba_kernel_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "ba_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "ba_get_timing": (C.c_int, [C.c_void_p, C.POINTER(Timing)]),
    "ba_cost_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "ba_set_barrier_timeout": (C.c_int, [C.c_void_p, C.c_int64]),
    "ba_debug_checks": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                                  C.POINTER(C.c_uint32), C.POINTER(C.c_int64)]),
    "ba_probe_fp64_fma": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "ba_get_series_trace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    "ba_create_batch": (C.c_int, [C.POINTER(ProblemDesc), C.c_int32, C.POINTER(Options),
                                  C.POINTER(C.c_void_p)]),
    "ba_get_batch_layout": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p]),
    "ba_get_series_state": (C.c_int, [C.c_void_p, C.POINTER(SeriesInfo)]),
    "ba_lm_step_batch": (C.c_int, [C.c_void_p, C.POINTER(StepInfo), C.POINTER(C.c_int32)]),
    "ba_lm_solve_batch": (C.c_int, [C.c_void_p, C.POINTER(StepInfo), C.POINTER(C.c_int32)]),
    "ba_cost_batch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ba_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ba_get_schedule": (C.c_int, [C.c_void_p, C.POINTER(Schedule)]),
    "ba_set_step_graph": (C.c_int, [C.c_void_p, C.c_int32]),
    "ba_get_step_graph": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "ba_set_schedule": (C.c_int, [C.c_void_p, C.POINTER(Schedule)]),
    "ba_adjoint": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_int32, C.POINTER(SeriesInfo)]),
    "ba_solve_schur_pcg": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32, C.c_double,
                                     C.c_int32, C.POINTER(PcgInfo)]),
    "ba_destroy": (C.c_int, [C.c_void_p]),
    "ba_status_string": (C.c_char_p, [C.c_int]),
    "ba_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str | None = None) -> C.CDLL:
    """Load libpoba.so (built in-tree by paper_2204_12834_gb300.build).  Raises when missing:
    there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    # POBA_CHECKS=1 selects the debug build with device-side index checks and buffer guards
    p = path or (CHECKS_LIB_PATH if os.environ.get("POBA_CHECKS") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise ImportError(f"libpoba.so not found at {p}; build it with "
                          "`python -m paper_2204_12834_gb300.build` (needs nvcc)")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib
