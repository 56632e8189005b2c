"""The ctypes structures of the binding have the C header's layout: a small C
program compiled against include/litevoxel.h prints sizeof and offsetof of
every field, and each must match ctypes (no GPU needed)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2511_02510_gb300 import litevoxel as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["lv_voxels", "lv_camera", "lv_raster_opts", "lv_fwd_out", "lv_prune_params", "lv_subdiv_params",
           "lv_aux_array", "lv_adam_params", "lv_lf_params", "lv_rows"]
# ctypes names that differ from the C field names (Python keywords)
C_NAME = {("lv_aux_array", "in_"): "in"}


def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "litevoxel.h"', "int main(void) {"]
    for sname in STRUCTS:
        lines.append(f'  printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in getattr(L, sname)._fields_:
            cname = C_NAME.get((sname, fname), fname)
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {cname}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True,
                       capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        s, f, v = line.split()
        res[(s, f)] = int(v)
    return res


def test_struct_layouts_match_the_header():
    lay = c_layout()
    for sname in STRUCTS:
        cls = getattr(L, sname)
        assert ctypes.sizeof(cls) == lay[(sname, "size")], sname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == lay[(sname, fname)], (sname, fname)
