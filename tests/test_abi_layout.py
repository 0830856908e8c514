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


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "gbstencil.h"

/* A plain C client: host-only calls of the ABI (no device is touched). */
int main(void) {
    double w[9];
    for (int i = 0; i < 9; i++) w[i] = 1.0 / 9.0;
    int64_t dims[2] = {100, 200};
    stencil_plan *plan = NULL;
    if (stencil_plan_create(&plan, STENCIL_BOX, 2, 1, w, STENCIL_F64, dims, 0) != STENCIL_OK) return 1;
    stencil_info info;
    if (stencil_plan_info(plan, &info) != STENCIL_OK) return 2;
    printf("path %d t %d K %d\n", info.path, info.t, info.K);
    if (stencil_plan_set_option(plan, "t", "3") != STENCIL_OK) return 3;
    if (stencil_plan_info(plan, &info) != STENCIL_OK || info.t != 3) return 4;
    if (stencil_plan_set_option(plan, "no_such_key", "1") != STENCIL_ERR_INVALID_ARG) return 5;
    if (strstr(stencil_last_error(), "no_such_key") == NULL) return 6;
    printf("ws %zu\n", stencil_plan_workspace_bytes(plan, 0));
    stencil_plan_destroy(plan);
    stencil_model_in q = {STENCIL_BOX, 2, 3, 1, 8, 0.4375, 1.0, 1.2586e12, 1.2586e12, 6.8e12};
    stencil_model_out o;
    if (stencil_model_predict(&q, &o) != STENCIL_OK) return 7;
    printf("alpha %.3f I_cu %.4f scenario %d\n", o.alpha, o.I_cu, o.scenario);
    printf("%s\n", stencil_status_string(STENCIL_ERR_UNSUPPORTED));
    return 0;
}
"""


def test_plain_c_client_links_and_runs():
    """A C11 program links libgbstencil.so with gcc (no C++ driver, no
    Python) and uses the host-only part of the ABI."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2603_00477_gb300 import build as gbuild
    lib = gbuild.build()
    libdir = os.path.dirname(lib)
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "client.c"), os.path.join(d, "client")
        with open(src, "w") as f:
            f.write(C_CLIENT)
        subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), src,
                               "-o", exe, "-L", libdir, "-lgbstencil", f"-Wl,-rpath,{libdir}"])
        res = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, (res.returncode, res.stdout, res.stderr)
    lines = res.stdout.splitlines()
    assert lines[0] == "path 1 t 1 K 9"  # FP64: CUDA cores, one step per sweep
    assert lines[1] == f"ws {102 * 202 * 8}"  # one stored FP64 grid: the ping-pong buffer
    assert lines[2] == "alpha 1.000 I_cu 6.1250 scenario 4"
    assert lines[3] == "unsupported"
