"""GPU parity of the tensor-core path (tcgen05 TF32 / TF32X3 / BF16X3 for FP32
grids, FP64 MMA for FP64 grids) against the FP64 oracle, through the C ABI.

Tolerances (normwise relative L-infinity over the interior): FP64 MMA 1e-12;
the FP32 forms within tc_bounds.tc_bound (operand rounding plus FP32
accumulation per MMA, summed over sweeps); the few-sweep cases below also
within the fixed values in TOL.
Dyadic weights on small integers (one step) are exact in every form and must
match bit for bit.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

from tc_bounds import tc_bound

pytestmark = pytest.mark.gpu

TOL = {"native64": 1e-12, "tf32x3": 1e-5, "bf16x3": 5e-5, "tf32": 3e-3, "f16": 3e-3, "f16x3": 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def tc_run(torch, shape, r, w, dims, u, steps, dtype, prec, t):
    plan = B.Plan(shape, 2, r, w, dtype, dims, t)
    if dtype == "f32":
        plan.set_option("precision", prec)
    plan.set_option("path", "tensor_core")
    info = plan.info()
    assert info["path"] == B.PATH_TENSOR_CORE and info["t"] == t
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    y = torch.full_like(x, float("nan"))
    plan.run(x, y, steps)
    B.stencil_device_status()
    out = y.cpu().numpy()
    plan.close()
    return out


def _interior(a, r, dims):
    return a[tuple(slice(r, r + n) for n in dims)]


CASES = [
    # shape, r, dims, steps, t, dtype, prec
    ("box", 1, (130, 140), 1, 1, "f32", "tf32"),
    ("box", 2, (257, 300), 4, 2, "f32", "tf32"),
    ("box", 2, (200, 131), 8, 4, "f32", "tf32x3"),
    ("box", 2, (129, 129), 3, 3, "f32", "bf16x3"),
    ("star", 2, (190, 260), 6, 3, "f32", "tf32x3"),
    ("star", 1, (128, 128), 7, 4, "f32", "bf16x3"),
    ("box", 3, (140, 75), 5, 2, "f32", "tf32x3"),     # remainder sweep t'=1
    ("box", 1, (5, 7), 3, 3, "f32", "tf32x3"),         # grid smaller than the band
    ("star", 6, (100, 100), 2, 2, "f32", "tf32x3"),    # R = 12
    ("box", 3, (131, 77), 6, 1, "f64", "native"),
    ("box", 3, (131, 77), 8, 4, "f64", "native"),
    ("star", 2, (70, 200), 6, 3, "f64", "native"),
    ("box", 1, (3, 300), 4, 2, "f64", "native"),
    ("box", 2, (257, 300), 4, 2, "f32", "f16"),
    ("box", 2, (200, 131), 8, 4, "f32", "f16"),        # R = 8
    ("star", 2, (190, 260), 6, 3, "f32", "f16"),
    ("box", 1, (130, 140), 1, 1, "f32", "f16x3"),
    ("box", 2, (300, 500), 5, 2, "f32", "f16x3"),      # remainder sweep t' = 1; more tiles than SMs
    ("box", 3, (140, 75), 5, 2, "f32", "f16x3"),       # R = 6, remainder sweep t' = 1
    ("star", 1, (128, 128), 7, 4, "f32", "f16x3"),
    ("box", 1, (5, 7), 3, 3, "f32", "f16"),            # grid smaller than the band
    # the wide FP16 kernel with more tiles than SMs (each persistent CTA
    # cycles through both operand buffers and accumulators several times)
    ("box", 2, (4000, 4000), 6, 2, "f32", "f16"),       # 16 x 32 tiles of 256 x 128
    ("star", 3, (3000, 3500), 8, 4, "f32", "f16"),      # R = 12: 128-row tiles
    ("box", 1, (2000, 3001), 9, 4, "f32", "f16x3"),     # R = 4, 128-row tiles, unaligned rows
    ("box", 2, (700, 900), 4, 4, "f32", "f16x3"),       # R = 8: 128-row tiles, one operand buffer
    # one operand buffer (hi + lo forms at R = 7 .. 12) with more tiles than
    # SMs: each CTA converts a tile only after the previous tile's MMAs
    ("box", 2, (2000, 2100), 8, 4, "f32", "bf16x3"),    # R = 8, 272 tiles
    ("box", 5, (2100, 1900), 4, 2, "f32", "f16x3"),     # R = 10, 10 K blocks
    ("star", 3, (1700, 2300), 8, 4, "f32", "bf16x3"),   # R = 12
    ("box", 7, (1000, 1000), 2, 1, "f32", "f16x3"),     # R = 7 without fusion
]


@pytest.mark.parametrize("shape,r,dims,steps,t,dtype,prec", CASES)
def test_tc_matches_oracle(torch, shape, r, dims, steps, t, dtype, prec):
    npdt = np.float64 if dtype == "f64" else np.float32
    w, u = inputs.problem(shape, 2, r, dims, seed=300 + r + t, dtype=npdt)
    rng = np.random.default_rng(11)  # non-zero halo: the band fix-up must keep it fixed
    mask = np.ones(u.shape, bool)
    mask[tuple(slice(r, r + n) for n in dims)] = False
    u[mask] = rng.uniform(0, 1, size=mask.sum()).astype(npdt)
    y = tc_run(torch, shape, r, w, dims, u, steps, dtype, prec, t)
    ref = oracle.run(shape, 2, r, w, dims, u.astype(np.float64), steps)
    err = oracle.rel_linf(_interior(y, r, dims), _interior(ref, r, dims))
    key = "native64" if dtype == "f64" else prec
    assert err <= TOL[key], (err, TOL[key])
    assert np.array_equal(y[mask], u[mask])
    assert not np.isnan(y).any()


@pytest.mark.parametrize("dtype,prec", [("f64", "native"), ("f32", "tf32"), ("f32", "tf32x3"), ("f32", "bf16x3"),
                                        ("f32", "f16"), ("f32", "f16x3")])
@pytest.mark.parametrize("shape,r", [("box", 3), ("star", 2), ("box", 1)])
def test_tc_dyadic_one_step_bitwise(torch, dtype, prec, shape, r):
    """Weights k/64 (k <= 8) and integer fields below 2^8 are exact in TF32 and
    BF16 and every partial sum fits FP32: the MMA result must be exact."""
    dims = (150, 203)
    rng = np.random.default_rng(17)
    K = inputs.num_weights(shape, 2, r)
    w = rng.integers(0, 9, size=K) / 64.0
    u = rng.integers(0, 256, size=(dims[0] + 2 * r, dims[1] + 2 * r)).astype(np.float64)
    npdt = np.float64 if dtype == "f64" else np.float32
    y = tc_run(torch, shape, r, w, dims, u.astype(npdt), 1, dtype, prec, 1)
    ref = oracle.run(shape, 2, r, w, dims, u, 1)
    assert np.array_equal(y.astype(np.float64), ref)


def test_tc_constant_field(torch):
    dims = (256, 256)
    w = inputs.weights("box", 2, 2, seed=3)
    u = np.full((260, 260), 0.75, dtype=np.float32)
    y = tc_run(torch, "box", 2, w, dims, u, 8, "f32", "tf32x3", 4)
    assert np.max(np.abs(y - 0.75)) <= 2e-6


@functools.lru_cache(maxsize=1)
def _big(shape, r, dims, seed, dtype):
    w, u = inputs.problem(shape, 2, r, dims, seed=seed, dtype=np.float64 if dtype == "f64" else np.float32)
    u.setflags(write=False)
    return w, u


SAMPLES = [((0, 0), (4, 4)), ((0, 8190), (3, 8194)), ((16380, 16379), (16384, 16384)), ((9000, 3), (9002, 7)),
           ((7000, 7000), (7003, 7005))]


@pytest.mark.parametrize("t", [1, 2, 3, 4])
def test_config_box2d3r_16384_fp64_mma_sampled(torch, t):
    """Box-2D3R FP64 on 16384^2, 100 steps, FP64 MMA path."""
    dims = (16384, 16384)
    w, u = _big("box", 3, dims, 2, "f64")
    y = _run_big(torch, "box", 3, w, dims, u, 100, "f64", "native", t)
    for lo, hi in SAMPLES:
        ref = oracle.run_region("box", 2, 3, w, dims, u, 100, lo, hi)
        got = y[lo[0] + 3:hi[0] + 3, lo[1] + 3:hi[1] + 3].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= 1e-12, (lo, hi)
    del y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec,t", [("tf32", 4), ("tf32x3", 2), ("bf16x3", 3), ("f16", 4), ("f16x3", 2)])
def test_config_box2d2r_16384_f32_sampled(torch, prec, t):
    """Box-2D2R FP32 on 16384^2 (smooth sine-mode field), 40 steps, sampled."""
    dims = (16384, 16384)
    w, u = inputs.problem("box", 2, 2, dims, seed=4, dtype=np.float32, field="sine")
    plan = B.Plan("box", 2, 2, w, "f32", dims, t)
    plan.set_option("precision", prec)
    plan.set_option("path", "tensor_core")
    bound = tc_bound(prec, 40, t, plan.handle, "box", 2)
    plan.close()
    y = _run_big(torch, "box", 2, w, dims, u, 40, "f32", prec, t)
    u64 = u.astype(np.float64)
    gots, refs = [], []
    for lo, hi in SAMPLES:
        refs.append(oracle.run_region("box", 2, 2, w, dims, u64, 40, lo, hi).ravel())
        gots.append(y[lo[0] + 2:hi[0] + 2, lo[1] + 2:hi[1] + 2].cpu().numpy().astype(np.float64).ravel())
    # normwise over the union of the sampled boxes
    err = oracle.rel_linf(np.concatenate(gots), np.concatenate(refs))
    assert err <= bound, (err, bound)
    del y
    torch.cuda.empty_cache()


def _run_big(torch, shape, r, w, dims, u, steps, dtype, prec, t):
    plan = B.Plan(shape, 2, r, w, dtype, dims, t)
    if dtype == "f32":
        plan.set_option("precision", prec)
    plan.set_option("path", "tensor_core")
    x = torch.from_numpy(np.array(u)).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, steps)
    B.stencil_device_status()
    plan.close()
    del x
    return y
