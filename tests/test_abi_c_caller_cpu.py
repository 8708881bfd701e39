"""libpoba from a plain C99 program (no Python, no torch): tests/cpp/abi_c_caller.c includes
only include/poba.h, links libpoba.so and exercises the entry points' host-side paths
(defaults, status strings, argument validation, error messages).  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_links_and_calls_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("needs a C compiler")
    from paper_2204_12834_gb300 import build as b
    b.build()
    libdir = os.path.join(ROOT, "paper_2204_12834_gb300")
    exe = tmp_path / "abi_c_caller"
    res = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                          "-I", os.path.join(ROOT, "include"),
                          os.path.join(ROOT, "tests", "cpp", "abi_c_caller.c"),
                          "-L", libdir, "-lpoba", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "0 failure(s)" in run.stdout
