"""stencil_run_noalloc: the multi-sweep run for callers that may not allocate
device memory (an application that owns all device memory through its own
allocator, or a loop that cannot take the implicit synchronisation of an
allocation).  Its ping-pong buffer is the library's static device array, so
no device memory is allocated by the call; checked against the CPU oracle and
against the ordinary stencil_run (caller-provided workspace) on two calls in
a row, on the CUDA-core, dense tensor-core and sparse tensor-core paths.
Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

from tc_bounds import sp_bound, tc_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def _interior(a, r, dims):
    return a[tuple(slice(r, r + n) for n in dims)]


# (shape, r, dims, steps, t, dtype, path, precision): every case takes more
# than one fused sweep, so the static array is used as the ping-pong buffer
CASES = [("box", 3, (600, 700), 7, 2, "f64", "auto", None),
         ("box", 2, (300, 452), 5, 2, "f32", "tensor_core", "tf32"),
         ("box", 2, (257, 300), 7, 3, "f32", "sparse_tensor_core", "tf32")]


@pytest.mark.parametrize("shape,r,dims,steps,t,dtype,path,prec", CASES)
def test_noalloc_matches_oracle_and_stencil_run_twice(torch, shape, r, dims, steps, t, dtype, path, prec):
    npdt = np.float64 if dtype == "f64" else np.float32
    w, u = inputs.problem(shape, 2, r, dims, seed=41, dtype=npdt)
    plan = B.Plan(shape, 2, r, w, dtype, dims, t)
    if prec:
        plan.set_option("precision", prec)
    if path != "auto":
        plan.set_option("path", path)
    if path == "tensor_core":
        tol = tc_bound(prec, steps, t, plan.handle, shape, r)
    elif path == "sparse_tensor_core":
        tol = sp_bound(plan.handle, shape, r, steps, t)
    else:
        tol = 1e-12
    ref = oracle.run(shape, 2, r, w, dims, u.astype(np.float64), steps)
    x = torch.from_numpy(u).cuda()
    y_ws = torch.empty_like(x)
    plan.run(x, y_ws, steps)
    torch.cuda.synchronize()
    with_ws = y_ws.cpu().numpy().astype(np.float64)
    ys = [torch.full_like(x, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for i, y in enumerate(ys):
        free0 = torch.cuda.mem_get_info()[0]
        B.stencil_run_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), steps)
        torch.cuda.synchronize()
        if i == 1:  # the first call may load the library's module; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
        got = y.cpu().numpy().astype(np.float64)
        assert not np.isnan(got).any()
        assert oracle.rel_linf(_interior(got, r, dims), _interior(ref, r, dims)) <= tol
        assert oracle.rel_linf(_interior(got, r, dims), _interior(with_ws, r, dims)) <= 2 * tol
    plan.close()


def test_noalloc_single_sweep_takes_any_size(torch):
    """A run of at most one fused sweep (steps <= t) uses no scratch, so a grid
    above the 64 MiB array runs; with more sweeps it is refused before any
    launch or memory access (the two addresses are only compared)."""
    dims = (4096, 4096)
    w, u = inputs.problem("box", 2, 3, dims, seed=43)
    plan = B.Plan("box", 2, 3, w, "f64", dims, 2)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    ref = torch.empty_like(x)
    plan.run(x, ref, 2)
    B.stencil_run_noalloc(plan.handle, x.data_ptr(), y.data_ptr(), 2)
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    n0 = B.stencil_launch_count()
    with pytest.raises(B.StencilError) as e:
        B.stencil_run_noalloc(plan.handle, 1 << 40, 1 << 41, 3)
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    assert B.stencil_launch_count() == n0
    plan.close()


def test_noalloc_refuses_host_buffers(torch):
    """in and out must be memory of the current device: a host buffer is
    refused before any launch."""
    dims = (64, 64)
    w, u = inputs.problem("box", 2, 3, dims, seed=44)
    plan = B.Plan("box", 2, 3, w, "f64", dims, 1)
    x = torch.from_numpy(u).cuda()
    h = torch.empty(tuple(x.shape), dtype=x.dtype)
    n0 = B.stencil_launch_count()
    with pytest.raises(B.StencilError) as e:
        B.stencil_run_noalloc(plan.handle, x.data_ptr(), h.data_ptr(), 3)
    assert e.value.status == B.STENCIL_ERR_INVALID_ARG
    assert B.stencil_launch_count() == n0
    plan.close()
