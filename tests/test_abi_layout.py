"""The ctypes mirrors of the ABI structs in binding.py have the size and
field offsets the C compiler gives the declarations in include/gbstencil.h
(a host C program compiled with gcc prints them; no GPU)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_2603_00477_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["stencil_peaks", "stencil_info", "stencil_model_in", "stencil_model_out", "stencil_tc_layout",
           "stencil_sptc_layout", "stencil_tune_result", "stencil_grid_desc", "stencil_batch_tune_result"]


@pytest.fixture(scope="module")
def c_layout():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gbstencil.h"', "int main(void) {"]
    for name in STRUCTS:
        ct = getattr(B, name)
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in ct._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0; }"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines))
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        out = subprocess.check_output([exe], text=True)
    res = {}
    for l in out.splitlines():
        name, key, val = l.split()
        res[(name, key)] = int(val)
    return res


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_struct_matches_c(c_layout, name):
    ct = getattr(B, name)
    assert ctypes.sizeof(ct) == c_layout[(name, "size")], name
    for field, _ in ct._fields_:
        assert getattr(ct, field).offset == c_layout[(name, field)], (name, field)
