"""The binding's ctypes structures have the layout of the C structures in
include/gradsim.h: a C program built from the header prints every size and
field offset, and each must equal the ctypes one (CPU only, gcc)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["gs_contact", "gs_mesh_desc", "gs_mesh_info", "gs_camera", "gs_raster_desc", "gs_rigid_desc",
           "gs_rigid_grads", "gs_air", "gs_grads", "gs_allocator", "gs_server_opts", "gs_query", "gs_result",
           "gs_server_stats", "gs_kernel_time"]


def _c_name(py_field):
    return py_field[:-1] if py_field.endswith("_") else py_field  # lambda_ -> lambda


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_layouts_match_the_header(tmp_path):
    from paper_2104_02646_gb300 import gradsim as gs
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gradsim.h"', 'int main(void) {']
    expected = {}
    for name in STRUCTS:
        cls = getattr(gs, name)
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        expected[f"{name} size"] = __import__("ctypes").sizeof(cls)
        for f in cls._fields_:
            fname = f[0]
            lines.append(f'    printf("{name}.{fname} %zu\\n", offsetof({name}, {_c_name(fname)}));')
            expected[f"{name}.{fname}"] = getattr(cls, fname).offset
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for ln in out.splitlines():
        key, val = ln.rsplit(" ", 1)
        got[key] = int(val)
    mismatched = {k: (got.get(k), v) for k, v in expected.items() if got.get(k) != v}
    assert not mismatched, mismatched
