"""The ctypes structures of the Python binding have the layout the C header
declares: size and the offset of every field, read from a program that the
host compiler builds against include/pm.h (no GPU, no library load)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(structs):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pm.h"', "int main(void) {"]
    for name, fields in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        name, field, val = ln.split()
        res[(name, field)] = int(val)
    return res


def test_binding_structs_match_the_header():
    import paper_2603_01122_gb300 as pm
    structs = {n: getattr(pm, n) for n in ("pm_model", "pm_grid", "pm_human", "pm_mppi")}
    fields = {n: [f[0] for f in s._fields_] for n, s in structs.items()}
    lay = _c_layout(fields)
    import ctypes
    for n, s in structs.items():
        assert lay[(n, "sizeof")] == ctypes.sizeof(s), n
        for f in fields[n]:
            assert lay[(n, f)] == getattr(s, f).offset, (n, f)
