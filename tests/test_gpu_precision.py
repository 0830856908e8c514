"""Error growth of every FP32-grid arithmetic form against the FP64 oracle on
the precision workload (Box-2D2R, smooth sine-mode field), every 100 steps up
to 1000, on a 2048^2 interior (the oracle evaluates every point).

FP32 CUDA-core arithmetic must stay within the FP32 tolerance 1e-5; the
tensor-core forms within their derived bounds (tests/tc_bounds.py).  The
measured table is printed (run with -s to see it)."""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

from tc_bounds import tc_bound

pytestmark = pytest.mark.gpu

DIMS = (2048, 2048)
CHECK = list(range(100, 1001, 100))


@pytest.fixture(scope="module")
def problem():
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    w, u = inputs.problem("box", 2, 2, DIMS, seed=4, dtype=np.float32, field="sine")
    ref = u.astype(np.float64)
    refs = {}
    for k in CHECK:
        ref = oracle.run("box", 2, 2, w, DIMS, ref, 100)
        refs[k] = ref[2:-2, 2:-2].copy()
    return w, u, refs


FORMS = [("cuda_core", "native", 2)] + [("tensor_core", p, t) for p in ("tf32", "tf32x3", "bf16x3", "f16", "f16x3")
                                         for t in (1, 2, 4)]


@pytest.mark.parametrize("path,prec,t", FORMS)
def test_error_growth(problem, path, prec, t):
    import torch
    w, u, refs = problem
    plan = B.Plan("box", 2, 2, w, "f32", DIMS, t)
    if prec != "native":
        plan.set_option("precision", prec)
    plan.set_option("path", path)
    x = torch.from_numpy(u.copy()).cuda()
    y = torch.empty_like(x)
    errs = []
    for k in CHECK:
        plan.run(x, y, 100)
        B.stencil_device_status()
        got = y.cpu().numpy().astype(np.float64)[2:-2, 2:-2]
        errs.append(oracle.rel_linf(got, refs[k]))
        x, y = y, x
    print(f"\n{path}/{prec}/t={t}: " + " ".join(f"{e:.2e}" for e in errs))
    for k, e in zip(CHECK, errs):
        if path == "cuda_core":
            assert e <= 1e-5, (k, e)
        else:
            # runs of 100 steps restart the fused schedule: 100 = q*t + rem
            per_run = tc_bound(prec, 100, t, plan.handle, "box", 2)
            assert e <= per_run * k / 100, (k, e, per_run)
    plan.close()
