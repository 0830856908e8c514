"""GPU parity of the staging variants the FP32 sweeps choose from: 16-byte
copies when every stored row is a multiple of 16 bytes and the buffers are
16-byte aligned (tile grid shifted so each staged window starts on a 16-byte
boundary), 4-byte copies otherwise.  Each case runs once on a grid whose
stored rows are 16-byte multiples and once from buffers that start 4 bytes
past a 16-byte boundary (forcing the 4-byte path), on every FP32 path, and
both results must match the oracle within the path's bound and each other."""
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


def _bound(path, prec, plan, shape, r, steps, t):
    if path == "cuda_core":
        return 1e-5
    if path == "sparse_tensor_core":
        return sp_bound(plan.handle, shape, r, steps, t)
    return tc_bound(prec, steps, t, plan.handle, shape, r)


def _run(torch, plan, u, steps, offset):
    """Run from buffers that start `offset` elements into a larger allocation."""
    n = u.size
    xb = torch.zeros(n + 8, dtype=torch.float32, device="cuda")
    yb = torch.full((n + 8,), float("nan"), dtype=torch.float32, device="cuda")
    x = xb[offset:offset + n].view(u.shape)
    y = yb[offset:offset + n].view(u.shape)
    x.copy_(torch.from_numpy(u))
    plan.ensure_workspace(x.device)
    B.stencil_run(plan.handle, x.data_ptr(), y.data_ptr(), steps)
    B.stencil_device_status()
    torch.cuda.synchronize()
    return y.cpu().numpy()


CASES = [
    # path, precision, shape, r, dims (ny, nx), steps, t   (stored row = nx + 2r)
    ("cuda_core", "native", "box", 2, (150, 296), 4, 1),      # 300: 16-byte rows
    ("cuda_core", "native", "star", 1, (97, 202), 5, 2),      # 204
    ("cuda_core", "native", "box", 3, (120, 258), 6, 3),      # 264
    ("tensor_core", "tf32", "box", 2, (140, 316), 4, 2),      # 320
    ("tensor_core", "tf32", "box", 2, (133, 252), 3, 3),      # 256, R = 6: shifted grid
    ("tensor_core", "tf32x3", "star", 1, (129, 198), 4, 1),   # 200, R = 1: shifted grid
    ("tensor_core", "f16", "box", 2, (140, 316), 4, 2),       # 320
    ("tensor_core", "f16x3", "box", 2, (133, 252), 3, 3),     # 256, R = 6
    ("sparse_tensor_core", "tf32", "box", 2, (200, 316), 3, 3),
    ("sparse_tensor_core", "tf32", "star", 3, (130, 250), 4, 2),
    ("sparse_tensor_core", "tf32", "box", 1, (77, 126), 3, 3),
]


@pytest.mark.parametrize("path,prec,shape,r,dims,steps,t", CASES)
def test_aligned_and_unaligned_staging_agree(torch, path, prec, shape, r, dims, steps, t):
    assert (dims[1] + 2 * r) % 4 == 0
    w, u = inputs.problem(shape, 2, r, dims, seed=700 + r + t, dtype=np.float32)
    plan = B.Plan(shape, 2, r, w, "f32", dims, t)
    if prec != "native":
        plan.set_option("precision", prec)
    plan.set_option("path", path)
    bound = _bound(path, prec, plan, shape, r, steps, t)
    ref = oracle.run(shape, 2, r, w, dims, u.astype(np.float64), steps)
    inner = tuple(slice(r, r + n) for n in dims)
    outs = []
    for offset in (0, 1):  # 16-byte aligned buffers, then 4 bytes past the boundary
        y = _run(torch, plan, u, steps, offset)
        assert not np.isnan(y).any()
        err = oracle.rel_linf(y[inner], ref[inner])
        assert err <= bound, (offset, err, bound)
        outs.append(y)
    plan.close()
    # both staging variants compute the same arithmetic
    if path == "cuda_core":
        assert np.array_equal(outs[0], outs[1])
    else:
        assert oracle.rel_linf(outs[0][inner], outs[1][inner]) <= 2 * bound
