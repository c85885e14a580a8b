"""The C header and the Python binding describe the same ABI (no GPU): a C99
program compiled against include/gs.h (gcc -std=c99 -pedantic, so the header
is plain C) prints the size and field offsets of every struct and the value of
every enumerator; the ctypes mirrors in the binding must match them."""
import ctypes
import json
import os
import shutil
import subprocess

import pytest

from paper_2501_06838_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {"gs_head": _abi.GsHead, "gs_gaussians": _abi.GsGaussians, "gs_view": _abi.GsView,
           "gs_stats": _abi.GsStats, "gs_peaks": _abi.GsPeaks, "gs_tuning": _abi.GsTuning}
ENUMS = ["GS_OK", "GS_ERR_INVALID", "GS_ERR_CAPACITY", "GS_ERR_CUDA", "GS_ERR_UNSUPPORTED",
         "GS_ERR_TIMEOUT", "GS_ERR_INTERNAL", "GS_F32", "GS_BF16", "GS_F16", "GS_NORM_DENSITY",
         "GS_NORM_PEAK", "GS_WINDOW_SIGMA", "GS_WINDOW_RATIO", "GS_ALIGN_EQ4", "GS_ALIGN_HALF",
         "GS_ADJOINT_AUTO", "GS_ADJOINT_TILE", "GS_ADJOINT_GAUSSIAN", "GS_ADJOINT_QUADRANT",
         "GS_BINNING_AUTO", "GS_BINNING_SORT", "GS_BINNING_GRID"]


def _program() -> str:
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"',
             'int main(void) {', '  printf("{");']
    first = True
    for name, cls in STRUCTS.items():
        for key, expr in [(f"{name}", f"sizeof({name})")] + \
                [(f"{name}.{f}", f"offsetof({name}, {f})") for f, _ in cls._fields_]:
            sep = "" if first else ", "
            first = False
            lines.append(f'  printf("{sep}\\"{key}\\": %lu", (unsigned long)({expr}));')
    for e in ENUMS:
        lines.append(f'  printf(", \\"{e}\\": %d", (int)({e}));')
    lines += ['  printf("}\\n");', '  return 0;', '}']
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text(_program())
    subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layout_matches_header(layout, name):
    cls = STRUCTS[name]
    assert ctypes.sizeof(cls) == layout[name], name
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == layout[f"{name}.{f}"], f"{name}.{f}"


def test_enumerators_match_header(layout):
    for e in ENUMS:
        assert getattr(_abi, e) == layout[e], e
