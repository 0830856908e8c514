"""stencil_host_alloc: page-locked host buffers on 2 MiB pages for
stencil_run_host; the run from them equals the device-resident run."""
import numpy as np
import pytest

from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_run_host_from_huge_page_buffers():
    import torch

    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    dims = (300, 500)
    w, u = inputs.problem("box", 2, 3, dims, seed=61)
    plan = B.Plan("box", 2, 3, w, "f64", dims, 1)
    h_in = B.host_empty(u.shape, "f64")
    h_out = B.host_empty(u.shape, "f64")
    assert h_in.data_ptr() % (2 << 20) == 0 and h_out.data_ptr() % (2 << 20) == 0
    assert float(h_out.abs().max()) == 0.0  # zero-filled
    h_in.copy_(torch.from_numpy(u))
    plan.run_host(h_in, h_out, 6)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 6)
    torch.cuda.synchronize()
    assert torch.equal(h_out, y.cpu())
    plan.close()
    ptr = B.stencil_host_alloc(1 << 20)
    B.stencil_host_free(ptr)
    with pytest.raises(B.StencilError):
        B.stencil_host_free(ptr)  # already released
