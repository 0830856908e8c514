"""stencil_run_noalloc: the multi-sweep run for callers that may not allocate
device memory (no cudaMalloc anywhere on the call), checked against the
ordinary stencil_run, which uses caller-provided workspace, on two calls in a
row.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_noalloc_matches_stencil_run_twice():
    import torch

    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    dims = (600, 700)
    w, u = inputs.problem("box", 2, 3, dims, seed=41)
    plan = B.Plan("box", 2, 3, w, "f64", dims, 2)  # 7 steps = 4 fused sweeps: the ping-pong buffer is used
    x = torch.from_numpy(u).cuda()
    ref = torch.empty_like(x)
    plan.run(x, ref, 7)
    torch.cuda.synchronize()
    ref_np = ref.cpu().numpy()
    scale = float(np.max(np.abs(ref_np)))
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        B.stencil_run_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), 7)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert float(np.max(np.abs(got - ref_np))) / scale <= 1e-12
    # a grid above the 64 MiB scratch is refused before any launch or access
    # (the two addresses are only compared, never dereferenced)
    big = B.Plan("box", 2, 3, w, "f64", (4096, 4096), 1)
    n0 = B.stencil_launch_count()
    with pytest.raises(B.StencilError) as e:
        B.stencil_run_noalloc(big.handle, 1 << 40, 1 << 41, 3)
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    assert B.stencil_launch_count() == n0
    big.close()
    plan.close()
