"""The ctypes mirrors of the C ABI structs match the header's layout (sizes
and field offsets as gcc lays them out), so no field is read from the wrong
place (CPU only)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["batmap_params", "batmap_info", "batmap_timing", "batmap_out", "batmap_serve_opts",
           "batmap_serve_stats"]


def _cuda_include():
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime_api.h")):
            return os.path.join(cand, "include")
    return None


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_1102_1003_gb300 import batmap as B
    inc = _cuda_include()
    if inc is None or shutil.which("gcc") is None:
        pytest.skip("gcc or the CUDA headers are missing")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "batmap.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(B, s)._fields_:
            lines.append(f'printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines))
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", inc, str(src),
                           "-o", str(exe)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = line.split()
        out[(s, f)] = int(v)
    return out


@pytest.mark.parametrize("name", STRUCTS)
def test_struct_layout_matches_header(c_layout, name):
    from paper_1102_1003_gb300 import batmap as B
    cls = getattr(B, name)
    assert ctypes.sizeof(cls) == c_layout[(name, "size")]
    for f, _ in cls._fields_:
        assert getattr(cls, f).offset == c_layout[(name, f)], f
