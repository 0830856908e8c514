"""GPU parity of the 2:4-structured sparse tensor-core path (mma.sp TF32,
paper Sec. 4.3) against the FP64 oracle, through the C ABI.

Tolerance (normwise relative L-infinity over the interior), derived like the
dense TF32 form's: per fused sweep the operands are rounded to TF32
(P = 2 * 2^-11) and every sparse MMA adds into an FP32 accumulator
(n_mma * 2^-23, n_mma = an upper bound of the sparse instructions per output
counted from the band geometry, tests/tc_bounds.py); with positive
weights summing to 1 the errors add over sweeps.  Dyadic weights on small
integers are exact and must match bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

from tc_bounds import sp_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def sp_run(torch, shape, r, w, dims, u, steps, t):
    plan = B.Plan(shape, 2, r, w, "f32", dims, t)
    plan.set_option("precision", "tf32")
    plan.set_option("path", "sparse_tensor_core")
    info = plan.info()
    assert info["path"] == B.PATH_SPARSE_TENSOR_CORE and info["t"] == t
    bound = sp_bound(plan.handle, shape, r, steps, t)
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    y = torch.full_like(x, float("nan"))
    n0 = B.stencil_launch_count()
    plan.run(x, y, steps)
    B.stencil_device_status()
    assert B.stencil_launch_count() > n0
    out = y.cpu().numpy()
    plan.close()
    return out, bound


def _interior(a, r, dims):
    return a[tuple(slice(r, r + n) for n in dims)]


CASES = [
    # shape, r, dims, steps, t
    ("box", 1, (130, 140), 1, 1),
    ("box", 2, (257, 300), 4, 2),
    ("box", 2, (200, 131), 8, 4),      # R = 8: three instructions per line
    ("box", 2, (129, 129), 3, 3),
    ("star", 2, (190, 260), 6, 3),
    ("star", 1, (128, 128), 7, 4),     # remainder sweep t' = 3
    ("box", 3, (140, 75), 5, 2),       # remainder sweep t' = 1
    ("box", 1, (5, 7), 3, 3),          # grid smaller than the band
    ("star", 6, (100, 100), 2, 2),     # R = 12: four instructions per line
    ("box", 3, (300, 211), 8, 4),      # R = 12, box
    ("box", 7, (90, 170), 1, 1),
]


@pytest.mark.parametrize("shape,r,dims,steps,t", CASES)
def test_sparse_matches_oracle(torch, shape, r, dims, steps, t):
    w, u = inputs.problem(shape, 2, r, dims, seed=500 + r + t, dtype=np.float32)
    rng = np.random.default_rng(13)  # non-zero halo: the band fix-up must keep it fixed
    mask = np.ones(u.shape, bool)
    mask[tuple(slice(r, r + n) for n in dims)] = False
    u[mask] = rng.uniform(0, 1, size=mask.sum()).astype(np.float32)
    y, bound = sp_run(torch, shape, r, w, dims, u, steps, t)
    ref = oracle.run(shape, 2, r, w, dims, u.astype(np.float64), steps)
    err = oracle.rel_linf(_interior(y, r, dims), _interior(ref, r, dims))
    assert err <= bound, (err, bound)
    assert np.array_equal(y[mask], u[mask])
    assert not np.isnan(y).any()


@pytest.mark.parametrize("shape,r", [("box", 3), ("star", 2), ("box", 1), ("box", 6)])
def test_sparse_dyadic_one_step_bitwise(torch, shape, r):
    """Weights k/64 (k <= 8) and integer fields below 2^8 are exact in TF32 and
    every partial sum fits FP32: the sparse MMA result must be exact."""
    dims = (150, 203)
    rng = np.random.default_rng(19)
    K = inputs.num_weights(shape, 2, r)
    w = rng.integers(0, 9, size=K) / 64.0
    u = rng.integers(0, 256, size=(dims[0] + 2 * r, dims[1] + 2 * r)).astype(np.float64)
    y, _ = sp_run(torch, shape, r, w, dims, u.astype(np.float32), 1, 1)
    ref = oracle.run(shape, 2, r, w, dims, u, 1)
    assert np.array_equal(y.astype(np.float64), ref)


SAMPLES = [((0, 0), (4, 4)), ((0, 8190), (3, 8194)), ((16380, 16379), (16384, 16384)), ((9000, 3), (9002, 7)),
           ((7000, 7000), (7003, 7005))]


@pytest.mark.parametrize("t", [1, 4])
def test_config_box2d2r_16384_sparse_sampled(torch, t):
    """Box-2D2R FP32 on 16384^2 (smooth sine-mode field), 40 steps, sampled."""
    dims = (16384, 16384)
    w, u = inputs.problem("box", 2, 2, dims, seed=4, dtype=np.float32, field="sine")
    plan = B.Plan("box", 2, 2, w, "f32", dims, t)
    plan.set_option("precision", "tf32")
    plan.set_option("path", "sparse_tensor_core")
    bound = sp_bound(plan.handle, "box", 2, 40, t)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 40)
    B.stencil_device_status()
    plan.close()
    del x
    u64 = u.astype(np.float64)
    gots, refs = [], []
    for lo, hi in SAMPLES:
        refs.append(oracle.run_region("box", 2, 2, w, dims, u64, 40, lo, hi).ravel())
        gots.append(y[lo[0] + 2:hi[0] + 2, lo[1] + 2:hi[1] + 2].cpu().numpy().astype(np.float64).ravel())
    err = oracle.rel_linf(np.concatenate(gots), np.concatenate(refs))
    assert err <= bound, (err, bound)
    del y
    torch.cuda.empty_cache()
