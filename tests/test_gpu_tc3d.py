"""GPU parity of 3-D FP32 grids on the FP16 tensor cores (tc3d_wide: one step
per sweep, the Toeplitz factor of each (dz, dy) line as the A operand, a ring
of staged input planes as the B operand) against the FP64 oracle, through the
C ABI.

Tolerance (normwise relative L-infinity over the interior), per sweep: the
FP16 rounding of the scaled field and weights (2 * 2^-11) plus one FP32
ulp per accumulation, with the accumulations per output counted here from
the stencil's lines (a box: (2r+1)^2 lines of half-width r; a star: line
(0, 0) of half-width r and 4r lines of half-width 0), each issuing the K
blocks of its 128 + 2r window that hold a non-zero column.  Dyadic weights on
small integer fields are exact and must match bit for bit.
"""
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


def line_halves(shape, r):
    if shape == "box":
        return [r] * (2 * r + 1) ** 2
    return [r] + [0] * (4 * r)


def bound(shape, r, sweeps):
    nkb = -(-(128 + 2 * r) // 16)
    n_mma = sum(min(nkb - 1, (r + h + 127) // 16) - (r - h) // 16 + 1 for h in line_halves(shape, r))
    return sweeps * (2.0 * 2 ** -11 + n_mma * 2 ** -23)


def run3d(torch, shape, r, w, dims, u, steps):
    plan = B.Plan(shape, 3, r, w, "f32", dims, 1)
    plan.set_option("precision", "f16")
    plan.set_option("path", "tensor_core")
    info = plan.info()
    assert info["path"] == B.PATH_TENSOR_CORE and info["t"] == 1
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    y = torch.full_like(x, float("nan"))
    plan.run(x, y, steps)
    B.stencil_device_status()
    out = y.cpu().numpy()
    plan.close()
    return out, info


CASES = [
    # shape, r, interior dims (z, y, x), steps
    ("box", 1, (20, 150, 260), 3),    # 2 x 3 tiles of 128 x 128 per plane, several runs
    ("star", 2, (17, 70, 124), 2),    # 64-row tiles, stored rows 16-byte multiples
    ("box", 2, (9, 40, 300), 2),      # 25 lines: 32-row tiles
    ("star", 3, (12, 65, 140), 2),    # R = 3: a ring of 8 planes
    ("star", 1, (1, 5, 7), 2),        # one plane, a grid smaller than a tile
    ("box", 1, (3, 130, 126), 1),     # the ring's first planes only; rows 16-byte multiples
]


@pytest.mark.parametrize("shape,r,dims,steps", CASES)
def test_tc3d_matches_oracle(torch, shape, r, dims, steps):
    w, u = inputs.problem(shape, 3, r, dims, seed=40 + r, dtype=np.float32)
    rng = np.random.default_rng(12)  # a non-zero halo: it must stay fixed
    mask = np.ones(u.shape, bool)
    mask[tuple(slice(r, r + n) for n in dims)] = False
    u[mask] = rng.uniform(0, 1, size=mask.sum()).astype(np.float32)
    y, info = run3d(torch, shape, r, w, dims, u, steps)
    ref = oracle.run(shape, 3, r, w, dims, u.astype(np.float64), steps)
    inner = tuple(slice(r, r + n) for n in dims)
    err = oracle.rel_linf(y[inner], ref[inner])
    assert err <= bound(shape, r, steps), (err, bound(shape, r, steps), info["tile"])
    assert np.array_equal(y[mask], u[mask])
    assert not np.isnan(y).any()


@pytest.mark.parametrize("shape,r", [("box", 1), ("star", 2)])
def test_tc3d_dyadic_one_step_bitwise(torch, shape, r):
    """Weights k/64 (k <= 8) and integer fields below 2^8 are exact in FP16
    (every plane tile then has the same power-of-two scale, so no weight is
    rescaled) and every partial sum fits FP32: the result must be exact."""
    dims = (7, 90, 150)
    rng = np.random.default_rng(19)
    K = inputs.num_weights(shape, 3, r)
    w = rng.integers(0, 9, size=K) / 64.0
    u = rng.integers(128, 256, size=tuple(n + 2 * r for n in dims)).astype(np.float64)
    y, _ = run3d(torch, shape, r, w, dims, u.astype(np.float32), 1)
    ref = oracle.run(shape, 3, r, w, dims, u, 1)
    assert np.array_equal(y.astype(np.float64), ref)


def test_tc3d_planes_of_different_scale(torch):
    """Planes whose magnitudes differ by 2^20 get different scales; the
    weights of each line are rescaled per output plane, so the normwise
    bound still holds."""
    shape, r, dims = "box", 1, (10, 60, 140)
    w, u = inputs.problem(shape, 3, r, dims, seed=5, dtype=np.float32)
    u[::2] *= np.float32(2.0 ** -20)
    y, _ = run3d(torch, shape, r, w, dims, u, 2)
    ref = oracle.run(shape, 3, r, w, dims, u.astype(np.float64), 2)
    inner = tuple(slice(r, r + n) for n in dims)
    assert oracle.rel_linf(y[inner], ref[inner]) <= bound(shape, r, 2)


def test_tc3d_unmet_wait_reports_timeout_then_recovers(torch):
    shape, r, dims = "box", 1, (6, 64, 128)
    w, u = inputs.problem(shape, 3, r, dims, seed=8, dtype=np.float32)
    plan = B.Plan(shape, 3, r, w, "f32", dims, 1)
    plan.set_option("precision", "f16")
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
    plan.run(x, y, 2)
    B.stencil_device_status()
    ref = oracle.run(shape, 3, r, w, dims, u.astype(np.float64), 2)
    assert oracle.rel_linf(y.cpu().numpy(), ref) <= bound(shape, r, 2)
    plan.close()
