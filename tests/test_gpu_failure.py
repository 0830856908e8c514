"""Failure detection without a GPU fault: bounded device waits forced to run
out (a dependency counter nothing increments; an mbarrier phase that never
completes), with a short limit.  The host must read STENCIL_ERR_TIMEOUT and
the CUDA context must stay usable for the next, normal run."""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def test_batch_unmet_dependency_times_out_then_recovers(torch):
    probs = []
    for i, (shape, r, ny, nx) in enumerate([("box", 1, 300, 200), ("star", 2, 100, 90)]):
        w, u = inputs.problem(shape, 2, r, (ny, nx), seed=700 + i, dtype=np.float32)
        probs.append((shape, r, ny, nx, w, u))
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 1)
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.empty_like(x) for x in ins]
    B.stencil_batch_set_option(batch.handle, "wait_cycles", 1 << 22)
    B.stencil_batch_set_option(batch.handle, "debug_block_sweep", 2)
    batch.run(ins, outs, 5)
    with pytest.raises(B.StencilError) as e:
        B.stencil_batch_status(batch.handle)
    assert e.value.status == B.STENCIL_ERR_TIMEOUT
    # same context, hook off: a normal run completes and is correct
    B.stencil_batch_set_option(batch.handle, "debug_block_sweep", -1)
    B.stencil_batch_set_option(batch.handle, "wait_cycles", 1 << 31)
    batch.run(ins, outs, 5)
    B.stencil_batch_status(batch.handle)
    for i, (shape, r, ny, nx, w, u) in enumerate(probs):
        ref = oracle.run(shape, 2, r, w, (ny, nx), u.astype(np.float64), 5)
        assert oracle.rel_linf(outs[i].cpu().numpy(), ref) <= 1e-5
    batch.close()


# tf32x3: tc2d_ws (256 + 4 stored columns: TMA staging); f16, f16x3, bf16x3:
# tc2d_wide, each with the normwise tolerance of its precision after 3 steps
TIMEOUT_FORMS = [("tf32x3", 1e-4), ("f16", 5e-3), ("f16x3", 1e-4), ("bf16x3", 1e-3)]


@pytest.mark.parametrize("prec,tol", TIMEOUT_FORMS)
def test_tensor_core_unmet_wait_reports_timeout_then_recovers(torch, prec, tol):
    dims = (256, 256)
    w, u = inputs.problem("box", 2, 2, dims, seed=9, dtype=np.float32)
    plan = B.Plan("box", 2, 2, w, "f32", dims, 1)
    plan.set_option("precision", prec)
    plan.set_option("path", "tensor_core")
    plan.set_option("debug_unmet_wait", 1)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 1)
    with pytest.raises(B.StencilError) as e:
        B.stencil_device_status()
    assert e.value.status == B.STENCIL_ERR_TIMEOUT
    B.stencil_device_status()  # the flag was cleared by the read
    plan.set_option("debug_unmet_wait", 0)
    plan.run(x, y, 3)
    B.stencil_device_status()
    ref = oracle.run("box", 2, 2, w, dims, u.astype(np.float64), 3)
    assert oracle.rel_linf(y.cpu().numpy(), ref) <= tol
    plan.close()
