"""GPU parity of FP64 grids on the FP16 tensor cores by exact splitting
(precision "ozaki") against the FP64 oracle, through the C ABI.

The split form claims FP64 accuracy: every digit product and every level sum
is exact (the host keeps each level's sum of absolute values below 2^24), so
the only roundings are the 53-bit cut of the input tile and of the weights
and the one conversion of the recombined integer.  The tolerance is the FP64
bar of every FP64 path, 1e-12 normwise relative L-infinity; dyadic inputs are
exact and must match bit for bit.
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


def split_plan(shape, r, w, dims, t):
    plan = B.Plan(shape, 2, r, w, "f64", dims, t)
    plan.set_option("precision", "ozaki")
    plan.set_option("path", "tensor_core")
    info = plan.info()
    assert info["path"] == B.PATH_TENSOR_CORE and info["precision"] == B.PREC_OZAKI and info["t"] == t
    return plan


def split_run(torch, shape, r, w, dims, u, steps, t):
    plan = split_plan(shape, r, w, dims, t)
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    y = torch.full_like(x, float("nan"))
    n0 = B.stencil_launch_count()
    plan.run(x, y, steps)
    B.stencil_device_status()
    assert B.stencil_launch_count() > n0
    out = y.cpu().numpy()
    plan.close()
    return out


def _interior(a, r, dims):
    return a[tuple(slice(r, r + n) for n in dims)]


CASES = [
    # shape, r, dims, steps, t: several 128 x 32 tiles with ragged tails,
    # remainders, fused radii up to 8, grids smaller than a tile or the band,
    # and grids of more tiles than CTAs (the double-buffered pipeline)
    ("box", 3, (300, 211), 3, 1),
    ("box", 3, (131, 77), 5, 1),
    ("box", 1, (257, 300), 7, 3),
    ("box", 2, (200, 131), 8, 3),      # R = 6, 169 taps: 8-bit digits (S = 7), one column block
    ("star", 1, (190, 260), 9, 4),     # remainder sweep t' = 1
    ("star", 2, (129, 129), 6, 2),
    ("star", 4, (140, 75), 4, 2),      # R = 8, one column block
    ("box", 1, (130, 140), 8, 4),
    ("box", 1, (5, 7), 3, 3),          # grid smaller than the band
    ("box", 3, (3, 300), 2, 1),        # three rows
    ("star", 3, (1, 1), 2, 1),         # one point
    ("box", 3, (640, 1600), 2, 1),     # 250 tiles: persistent CTAs take a second tile
    ("box", 1, (1024, 2048), 3, 3),    # 512 tiles, three to four per CTA
    ("box", 2, (600, 1000), 3, 3),     # 7-digit form over 315 tiles
]


@pytest.mark.parametrize("shape,r,dims,steps,t", CASES)
def test_split_matches_oracle(torch, shape, r, dims, steps, t):
    w, u = inputs.problem(shape, 2, r, dims, seed=900 + r + t, dtype=np.float64)
    rng = np.random.default_rng(23)  # non-zero halo: kept fixed, and read by the band sweep
    mask = np.ones(u.shape, bool)
    mask[tuple(slice(r, r + n) for n in dims)] = False
    u[mask] = rng.uniform(-1, 1, size=mask.sum())
    y = split_run(torch, shape, r, w, dims, u, steps, t)
    ref = oracle.run(shape, 2, r, w, dims, u, steps)
    err = oracle.rel_linf(_interior(y, r, dims), _interior(ref, r, dims))
    print(f"\nsplit {shape}-2D{r}R t={t} steps={steps} dims={dims}: rel_linf = {err:.2e}")
    assert err <= 1e-12, err
    assert np.array_equal(y[mask], u[mask])
    assert not np.isnan(y).any()


@pytest.mark.parametrize("shape,r", [("box", 3), ("star", 2), ("box", 1)])
def test_split_dyadic_one_step_bitwise(torch, shape, r):
    """Weights k/64 and integer fields below 2^8 have one non-zero digit each
    and an exact FP64 result: the split form must reproduce it bit for bit."""
    dims = (150, 203)
    rng = np.random.default_rng(29)
    K = inputs.num_weights(shape, 2, r)
    w = rng.integers(0, 9, size=K) / 64.0
    u = rng.integers(0, 256, size=(dims[0] + 2 * r, dims[1] + 2 * r)).astype(np.float64)
    y = split_run(torch, shape, r, w, dims, u, 1, 1)
    ref = oracle.run(shape, 2, r, w, dims, u, 1)
    assert np.array_equal(y, ref)


def test_split_signed_field_wide_range(torch):
    """Signed weights and a field spanning 30 binary orders of magnitude:
    the tile-relative fixed point keeps the normwise error at FP64 level."""
    dims = (260, 300)
    rng = np.random.default_rng(31)
    w = rng.uniform(-1, 1, size=49)
    u = rng.uniform(-1, 1, size=(dims[0] + 6, dims[1] + 6)) * np.exp2(rng.integers(-30, 1, size=(dims[0] + 6,
                                                                                              dims[1] + 6)))
    y = split_run(torch, "box", 3, w, dims, u, 4, 1)
    ref = oracle.run("box", 2, 3, w, dims, u, 4)
    err = oracle.rel_linf(_interior(y, 3, dims), _interior(ref, 3, dims))
    assert err <= 1e-12, err


def test_split_large_digits_sum_exactly(torch):
    """Digits chosen to drive the leading level sums up: every input digit of
    the staged tile is +-255 with the sign of the weight digit it meets at one
    output, so S_0 = sum_k |a_0 b_0| is as large as the weights allow.  An
    accumulator that dropped low bits would show at 2^-23 relative."""
    dims = (128, 32)
    R = 3
    rng = np.random.default_rng(37)
    w = rng.uniform(0.5, 1.0, size=49)
    w /= w.sum()
    # field: one value per stored cell with top digit +-255 (|u| in [2^-1, 1))
    signs = np.where(rng.random((dims[0] + 6, dims[1] + 6)) < 0.5, -1.0, 1.0)
    u = signs * (255 * 2.0 ** -8 + rng.integers(0, 2 ** 44, size=signs.shape) * 2.0 ** -53)
    # every weight is positive: at output (64, 16) make the 49 inputs positive
    u[64:64 + 7, 16:16 + 7] = np.abs(u[64:64 + 7, 16:16 + 7])
    y = split_run(torch, "box", R, w, dims, u, 1, 1)
    ref = oracle.run("box", 2, R, w, dims, u, 1)
    err = oracle.rel_linf(_interior(y, R, dims), _interior(ref, R, dims))
    assert err <= 1e-14, err  # the oracle's own 49-term FP64 sums; a dropped accumulator bit is ~1e-7


def test_split_nan_input_propagates(torch):
    """A NaN in the input makes every output the oracle marks NaN NaN (the
    split form marks its whole tile); the other outputs stay finite or NaN."""
    dims = (300, 100)
    w, u = inputs.problem("box", 2, 1, dims, seed=41, dtype=np.float64)
    u[150, 50] = np.nan
    y = split_run(torch, "box", 1, w, dims, u, 1, 1)
    ref = oracle.run("box", 2, 1, w, dims, u, 1)
    assert np.isnan(y[np.isnan(ref)]).all()
    fin = ~np.isnan(y) & ~np.isnan(ref)
    assert oracle.rel_linf(y[fin], ref[fin]) <= 1e-12


def test_split_agrees_with_fp64_cuda_cores(torch):
    dims = (513, 390)
    w, u = inputs.problem("box", 2, 3, dims, seed=43, dtype=np.float64)
    y = split_run(torch, "box", 3, w, dims, u, 20, 1)
    plan = B.Plan("box", 2, 3, w, "f64", dims, 1)
    plan.set_option("path", "cuda_core")
    x = torch.from_numpy(u).cuda()
    z = torch.empty_like(x)
    plan.run(x, z, 20)
    plan.close()
    err = oracle.rel_linf(_interior(y, 3, dims), _interior(z.cpu().numpy(), 3, dims))
    assert err <= 1e-13, err


SAMPLES = [((0, 0), (4, 4)), ((0, 8190), (3, 8194)), ((16380, 16379), (16384, 16384)), ((9000, 3), (9002, 7)),
           ((7000, 7000), (7003, 7005))]


def test_config_box2d3r_16384_split_sampled(torch):
    """Box-2D3R FP64 on 16384^2, 100 steps, split form, sampled boxes against
    the oracle's dependency-cone evaluation."""
    dims = (16384, 16384)
    w, u = inputs.problem("box", 2, 3, dims, seed=2, dtype=np.float64)
    plan = split_plan("box", 3, w, dims, 1)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.ensure_workspace(x.device)
    plan.run(x, y, 100)
    B.stencil_device_status()
    plan.close()
    del x
    for lo, hi in SAMPLES:
        ref = oracle.run_region("box", 2, 3, w, dims, u, 100, lo, hi)
        got = y[lo[0] + 3:hi[0] + 3, lo[1] + 3:hi[1] + 3].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= 1e-12, (lo, hi)
    del y
    torch.cuda.empty_cache()


def test_split_unmet_wait_reports_timeout_then_recovers(torch):
    dims = (256, 256)
    w, u = inputs.problem("box", 2, 3, dims, seed=47, dtype=np.float64)
    plan = split_plan("box", 3, w, dims, 1)
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
    ref = oracle.run("box", 2, 3, w, dims, u, 3)
    assert oracle.rel_linf(y.cpu().numpy(), ref) <= 1e-12
    plan.close()
