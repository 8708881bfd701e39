"""Build libpoba.so in-tree with nvcc for sm_103a (no torch, no cmake).

Each translation unit compiles in parallel to paper_2204_12834_gb300/_build/*.o and is linked
into paper_2204_12834_gb300/libpoba.so.  Objects are rebuilt when a source or header is newer.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpoba.so")
# the debug build: device-side index checks and buffer guards (csrc/checks.cuh)
BUILD_CHECKS = os.path.join(PKG, "_build_checks")
LIB_CHECKS = os.path.join(PKG, "libpoba_checks.so")
SOURCES = ["schedule.cpp", "kernels_linearize.cu", "kernels_series.cu", "kernels_persistent.cu",
           "kernels_adjoint.cu", "kernels_pcg.cu",
           "api.cu", "noalloc.cu", "probe.cu"]
HEADERS = [os.path.join(CSRC, "poba_internal.cuh"), os.path.join(CSRC, "tile_common.cuh"),
           os.path.join(CSRC, "checks.cuh"),
           os.path.join(CSRC, "jacobian_io.cuh"),
           os.path.join(CSRC, "series_body.cuh"),
           os.path.join(ROOT, "include", "poba.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpoba")
    return exe


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + HEADERS)


def _compile(src_name: str, extra: list[str], verbose: bool, build_dir: str = BUILD,
             defines: list[str] | None = None) -> str:
    src = os.path.join(CSRC, src_name)
    obj = os.path.join(build_dir, src_name.rsplit(".", 1)[0] + ".o")
    if _stale(obj, src) or extra:
        cmd = [nvcc(), "-c", src, "-o", obj] + FLAGS + (defines or []) + extra
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src_name}:\n{res.stdout}\n{res.stderr}")
        if extra and res.stderr:
            sys.stderr.write(res.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checks: bool = False) -> str:
    """Compile and link libpoba.so (checks: the debug build libpoba_checks.so, compiled with
    -DPOBA_CHECKS); returns its path."""
    build_dir, lib_path = (BUILD_CHECKS, LIB_CHECKS) if checks else (BUILD, LIB)
    defines = ["-DPOBA_CHECKS"] if checks else []
    os.makedirs(build_dir, exist_ok=True)
    if force:
        for f in os.listdir(build_dir):
            if f.endswith(".o"):
                os.remove(os.path.join(build_dir, f))
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, verbose, build_dir, defines), SOURCES))
    out = lib_path
    if force or not os.path.exists(out) or any(os.path.getmtime(o) > os.path.getmtime(out) for o in objs):
        tmp = out + ".tmp"
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "-ldl"]
        if verbose:
            print(" ".join(cmd), flush=True)
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
