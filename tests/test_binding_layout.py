"""The ctypes mirrors of the C-ABI structs in the Python binding have the
same size and field offsets as the structs include/nsl.h declares, as the
host C compiler lays them out.  CPU only (gcc, no GPU)."""
import ctypes as C
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["nsl_grid_desc", "nsl_camera", "nsl_light", "nsl_march_opts", "nsl_plume", "nsl_server_opts", "nsl_peaks",
           "nsl_train_opts",
           "nsl_server_stats"]


def _ctypes_layout():
    from paper_2604_03748_gb300 import nsl
    out = {}
    for name in STRUCTS:
        cls = getattr(nsl, name)
        out[name] = (C.sizeof(cls), {f[0]: getattr(cls, f[0]).offset for f in cls._fields_})
    return out


def test_struct_layouts_match_the_header(tmp_path):
    layout = _ctypes_layout()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nsl.h"', "int main(void) {"]
    for name, (_, fields) in layout.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0 and "not found" in r.stderr:
        pytest.skip("no host C compiler")
    assert r.returncode == 0, r.stderr
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for name, (size, fields) in layout.items():
        assert got[(name, "size")] == size, name
        for f, off in fields.items():
            assert got[(name, f)] == off, (name, f)
