"""The Python binding's ctypes mirrors of the C ABI structs have the layout the C compiler gives
include/poba.h: the same size and the same offset for every field, the same enum values, and
for every declared function the same number of parameters.  A small C program compiled against
the header prints sizeof / offsetof; no GPU and no library call is involved."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2204_12834_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# ctypes class -> C type name (ctypes field names drop a trailing "_" that avoids a keyword)
STRUCTS = {
    _lib.ProblemDesc: "ba_problem_desc",
    _lib.Options: "ba_options",
    _lib.SeriesInfo: "ba_series_info",
    _lib.StepInfo: "ba_step_info",
    _lib.PcgInfo: "ba_pcg_info",
    _lib.Timing: "ba_timing",
    _lib.Schedule: "ba_schedule",
}


def c_field(name: str) -> str:
    return name[:-1] if name.endswith("_") else name


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("needs a C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "poba.h"', "int main(void) {"]
    for cls, cname in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname} {c_field(f)} %zu\\n", offsetof({cname}, {c_field(f)}));')
    lines.append('  printf("BA_TIMING_CLASSES %d\\n", (int)BA_TIMING_CLASSES);')
    for code, name in _lib.STATUS_NAMES.items():
        lines.append(f'  printf("{name} %d\\n", (int){name});')
    lines.append('  printf("BA_FP64 %d\\nBA_FP32_BULK %d\\n", (int)BA_FP64, (int)BA_FP32_BULK);')
    lines.append("  return 0;\n}")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    res = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    table = {}
    for line in out.splitlines():
        *key, val = line.split()
        table[" ".join(key)] = int(val)
    return table


@pytest.mark.parametrize("cls", list(STRUCTS), ids=lambda c: c.__name__)
def test_struct_layout_matches_the_header(c_layout, cls):
    cname = STRUCTS[cls]
    assert C.sizeof(cls) == c_layout[f"{cname} size"], cname
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c_layout[f"{cname} {c_field(f)}"], (cname, f)


def test_enums_and_counts_match_the_header(c_layout):
    for code, name in _lib.STATUS_NAMES.items():
        assert c_layout[name] == code, name
    assert c_layout["BA_FP64"] == _lib.BA_FP64 and c_layout["BA_FP32_BULK"] == _lib.BA_FP32_BULK
    assert c_layout["BA_TIMING_CLASSES"] == len(_lib.TIMING_CLASSES)


def header_prototypes():
    """name -> number of parameters, for every function declared in include/poba.h."""
    import re
    text = open(os.path.join(ROOT, "include", "poba.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(?:ba_status|const char\s*\*)\s*(ba_\w+)\s*\(([^)]*)\)\s*;", text):
        params = m.group(2).strip()
        protos[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return protos


def test_binding_signatures_have_the_header_arity():
    protos = header_prototypes()
    assert len(protos) >= 30
    assert set(protos) == set(_lib.SIGNATURES)
    for name, n in protos.items():
        assert len(_lib.SIGNATURES[name][1]) == n, name
