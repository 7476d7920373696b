"""The ctypes mirror of include/lbm.h has every field of every public struct at the C compiler's
offset (gcc compiles a probe that prints offsetof for each field the binding declares)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1912_02018_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"lbm_domain": N.Domain, "lbm_cylinder": N.Cylinder, "lbm_params": N.Params, "lbm_init": N.Init,
           "lbm_window_grad": N.WindowGrad, "lbm_allocator": N.Allocator, "lbm_info_t": N.Info}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_fields_sit_at_the_c_offsets():
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lbm.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, fname, v = line.split()
        got[(cname, fname)] = int(v)
    for cname, py in STRUCTS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
