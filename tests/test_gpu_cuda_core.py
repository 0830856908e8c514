"""GPU parity of the CUDA-core path against the FP64 oracle, through the C ABI.

Tolerances (normwise relative L-infinity over the interior, max|g-o|/max|o|):
1e-12 for FP64 grids and 1e-5 for FP32 grids.  Exact special cases (dyadic
weights on small integers, one step) must match bit for bit.
"""
import functools

import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def _to_dev(torch, u, dtype):
    return torch.from_numpy(np.ascontiguousarray(u.astype(np.float64 if dtype == "f64" else np.float32))).cuda()


def gpu_run(torch, shape, d, r, w, dims, u, steps, dtype, t, tile=None, path="cuda_core"):
    plan = B.Plan(shape, d, r, w, dtype, dims, t)
    plan.set_option("path", path)
    if tile:
        plan.set_option("tile", tile)
    x = _to_dev(torch, u, dtype)
    y = torch.full_like(x, float("nan"))
    plan.run(x, y, steps)
    torch.cuda.synchronize()
    info = plan.info()
    plan.close()
    return x.cpu().numpy(), y.cpu().numpy(), info


@functools.lru_cache(maxsize=2)
def _big_problem(shape, d, r, dims, seed, dtype):
    w, u = inputs.problem(shape, d, r, dims, seed=seed, dtype=np.float64 if dtype == "f64" else np.float32)
    u.setflags(write=False)
    return w, u


def _interior(a, r, dims):
    return a[tuple(slice(r, r + n) for n in dims)]


CASES_2D = [
    # shape, r, dims, steps, t, dtype, tile
    ("star", 1, (150, 203), 5, 1, "f64", None),
    ("box", 1, (150, 203), 7, 3, "f64", None),
    ("box", 3, (131, 77), 6, 4, "f64", None),
    ("box", 3, (131, 77), 5, 2, "f64", None),          # remainder sweep (5 = 2+2+1)
    ("star", 2, (64, 64), 4, 2, "f32", None),
    ("box", 2, (129, 257), 9, 4, "f32", None),
    ("box", 2, (129, 257), 3, 1, "f32", None),
    ("star", 3, (97, 1), 4, 1, "f64", None),            # one column
    ("box", 1, (1, 1), 3, 2, "f64", None),              # one point
    ("star", 7, (45, 300), 2, 1, "f32", None),          # r = 7
    ("box", 7, (40, 41), 3, 2, "f64", None),
    ("box", 5, (33, 70), 4, 3, "f32", None),
    ("star", 4, (200, 90), 5, 2, "f64", "16x32"),       # small tiles, many CTAs
    ("box", 2, (7, 3), 4, 4, "f32", None),              # extent below r*t
    # FP32, r <= 2, grids of several whole interior tiles: the fixed-strip
    # sub-step (strips of 8 and 4 rows, all four window phases over t)
    ("box", 1, (300, 700), 5, 3, "f32", None),
    ("star", 1, (260, 600), 6, 2, "f32", None),
    ("star", 2, (300, 520), 7, 4, "f32", None),
    ("box", 2, (200, 600), 5, 2, "f32", None),
    ("box", 2, (170, 530), 3, 3, "f32", "42x128"),     # strips overlap (ch not a multiple of 4)
    ("box", 1, (99, 1030), 2, 1, "f32", None),
    # FP32, r >= 3: strips of 2 rows on whole interior tiles (64 x 128)
    ("box", 3, (300, 530), 3, 1, "f32", None),
    ("box", 7, (200, 300), 2, 1, "f32", None),
    ("star", 5, (260, 400), 3, 2, "f32", None),
    ("box", 4, (300, 301), 2, 2, "f32", None),          # unaligned rows
    ("star", 7, (150, 390), 2, 1, "f32", None),
]


@pytest.mark.parametrize("shape,r,dims,steps,t,dtype,tile", CASES_2D)
def test_2d_matches_oracle(torch, shape, r, dims, steps, t, dtype, tile):
    w, u = inputs.problem(shape, 2, r, dims, seed=100 + r, dtype=np.float64 if dtype == "f64" else np.float32)
    # a non-zero halo checks that the boundary stays fixed
    rng = np.random.default_rng(7)
    mask = np.ones(u.shape, bool)
    mask[tuple(slice(r, r + n) for n in dims)] = False
    u[mask] = rng.uniform(0, 1, size=mask.sum()).astype(u.dtype)
    x, y, info = gpu_run(torch, shape, 2, r, w, dims, u, steps, dtype, t, tile)
    assert info["t"] == t
    ref = oracle.run(shape, 2, r, w, dims, u.astype(np.float64), steps)
    err = oracle.rel_linf(_interior(y, r, dims), _interior(ref, r, dims))
    assert err <= TOL[dtype], err
    assert np.array_equal(y[mask], u[mask])          # halo copied unchanged
    assert np.array_equal(x, u)                      # input untouched


CASES_3D = [
    ("star", 1, (20, 33, 70), 4, 1, "f64"),
    ("star", 2, (19, 18, 45), 5, 2, "f64"),
    ("box", 1, (17, 23, 40), 3, 2, "f32"),
    ("box", 2, (12, 20, 37), 3, 1, "f64"),
    ("box", 2, (12, 20, 37), 4, 2, "f32"),
    ("star", 4, (13, 11, 33), 2, 1, "f32"),
    # FP32, t = 1, rotating partial sums along z: ragged tiles, runs of planes
    # per tile, unaligned rows (stored width not a multiple of 4), radius 3
    ("star", 1, (70, 45, 130), 3, 1, "f32"),
    ("star", 2, (41, 100, 201), 5, 1, "f32"),
    ("star", 3, (40, 37, 90), 2, 1, "f32"),
    ("box", 1, (150, 33, 70), 4, 1, "f32"),
    ("box", 1, (3, 5, 7), 2, 1, "f32"),
    ("star", 3, (1, 5, 9), 3, 2, "f64"),
]


@pytest.mark.parametrize("shape,r,dims,steps,t,dtype", CASES_3D)
def test_3d_matches_oracle(torch, shape, r, dims, steps, t, dtype):
    w, u = inputs.problem(shape, 3, r, dims, seed=200 + r, dtype=np.float64 if dtype == "f64" else np.float32)
    x, y, info = gpu_run(torch, shape, 3, r, w, dims, u, steps, dtype, t)
    ref = oracle.run(shape, 3, r, w, dims, u.astype(np.float64), steps)
    err = oracle.rel_linf(_interior(y, r, dims), _interior(ref, r, dims))
    assert err <= TOL[dtype], err


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,d,r,dims", [("box", 2, 3, (70, 131)), ("star", 3, 2, (9, 17, 36))])
def test_dyadic_one_step_bitwise(torch, dtype, shape, d, r, dims):
    rng = np.random.default_rng(5)
    K = inputs.num_weights(shape, d, r)
    w = rng.integers(0, 9, size=K) / 64.0
    u = rng.integers(0, 256, size=tuple(n + 2 * r for n in dims)).astype(np.float64)
    _, y, _ = gpu_run(torch, shape, d, r, w, dims, u, 1, dtype, 1)
    ref = oracle.run(shape, d, r, w, dims, u, 1)
    assert np.array_equal(y.astype(np.float64), ref)


def test_identity_and_shift_bitwise(torch):
    dims = (50, 77)
    _, u = inputs.problem("box", 2, 1, dims, seed=9)
    w = np.zeros(9)
    w[4] = 1.0
    _, y, _ = gpu_run(torch, "box", 2, 1, w, dims, u, 6, "f64", 3)
    assert np.array_equal(y, u)
    w = np.zeros(9)
    w[5] = 1.0  # offset (0, +1)
    _, y, _ = gpu_run(torch, "box", 2, 1, w, dims, u, 4, "f64", 2)
    ref = oracle.run("box", 2, 1, w, dims, u, 4)
    assert np.array_equal(y, ref)


def test_steps_zero_copies_input(torch):
    w, u = inputs.problem("star", 2, 2, (33, 40), seed=3)
    _, y, _ = gpu_run(torch, "star", 2, 2, w, (33, 40), u, 0, "f64", 1)
    assert np.array_equal(y, u)


def test_split_run_equals_single_run(torch):
    """Checkpoint/resume: 7 steps in one call equal 3 + 4 steps in two calls
    (the fused-sweep schedule restarts at the second call)."""
    dims = (90, 111)
    w, u = inputs.problem("box", 2, 2, dims, seed=4, dtype=np.float32)
    _, y7, _ = gpu_run(torch, "box", 2, 2, w, dims, u, 7, "f32", 2)
    _, y3, _ = gpu_run(torch, "box", 2, 2, w, dims, u, 3, "f32", 2)
    _, y34, _ = gpu_run(torch, "box", 2, 2, w, dims, y3, 4, "f32", 2)
    ref = oracle.run("box", 2, 2, w, dims, u.astype(np.float64), 7)
    assert oracle.rel_linf(_interior(y34, 2, dims), _interior(ref, 2, dims)) <= 1e-5
    # 7 = 2+2+2+1 versus 3 = 2+1 then 4 = 2+2: same steps, different fusion
    assert oracle.rel_linf(_interior(y34, 2, dims), _interior(y7, 2, dims)) <= 1e-5


def test_constant_field_preserved_on_gpu(torch):
    dims = (64, 96)
    w = inputs.weights("box", 2, 3, seed=6)
    u = np.full((70, 102), 0.625)
    _, y, _ = gpu_run(torch, "box", 2, 3, w, dims, u, 20, "f64", 4)
    assert np.max(np.abs(y - 0.625)) <= 2e-14


def test_host_io_entry_point(torch):
    dims = (100, 120)
    w, u = inputs.problem("box", 2, 1, dims, seed=8)
    plan = B.Plan("box", 2, 1, w, "f64", dims, 2)
    h_in = torch.from_numpy(u.copy()).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    plan.run_host(h_in, h_out, 5)
    ref = oracle.run("box", 2, 1, w, dims, u, 5)
    assert oracle.rel_linf(_interior(h_out.numpy(), 1, dims), _interior(ref, 1, dims)) <= 1e-12
    plan.close()


# ---- full-size configurations -------------------------------------------------------

def test_config_star2d1r_512_full(torch):
    """Star-2D1R FP64, 512^2 interior, zero halo, 10 steps, t = 1 (whole grid)."""
    dims = (512, 512)
    w, u = inputs.problem("star", 2, 1, dims, seed=1)
    _, y, info = gpu_run(torch, "star", 2, 1, w, dims, u, 10, "f64", 0, path="auto")
    ref = oracle.run("star", 2, 1, w, dims, u, 10)
    assert oracle.rel_linf(y, ref) <= 1e-12
    assert info["t"] == 1


SAMPLE_BOXES_2D = [((0, 0), (4, 4)), ((0, 8190), (3, 8194)), ((16380, 16379), (16384, 16384)),
                   ((9000, 3), (9002, 7))]


@pytest.mark.parametrize("t", [1, 2, 3, 4])
def test_config_box2d3r_16384_sampled(torch, t):
    """Box-2D3R FP64 on 16384^2, 100 steps: sampled outputs (corners, an edge,
    the middle) against the oracle's dependency-cone evaluation."""
    dims = (16384, 16384)
    w, u = _big_problem("box", 2, 3, dims, 2, "f64")
    plan = B.Plan("box", 2, 3, w, "f64", dims, t)
    plan.set_option("path", "cuda_core")
    x = torch.from_numpy(np.array(u)).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 100)
    torch.cuda.synchronize()
    for lo, hi in SAMPLE_BOXES_2D:
        ref = oracle.run_region("box", 2, 3, w, dims, u, 100, lo, hi)
        got = y[lo[0] + 3:hi[0] + 3, lo[1] + 3:hi[1] + 3].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= 1e-12, (lo, hi)
    plan.close()
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("t", [1, 2, 3, 4])
def test_config_box2d2r_f32_16384_cuda_core_sampled(torch, t):
    """Box-2D2R FP32 on 16384^2 (sine-mode field), 20 steps on CUDA cores:
    sampled outputs against the oracle's dependency-cone evaluation."""
    dims = (16384, 16384)
    w, u = inputs.problem("box", 2, 2, dims, seed=4, dtype=np.float32, field="sine")
    plan = B.Plan("box", 2, 2, w, "f32", dims, t)
    plan.set_option("path", "cuda_core")
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 20)
    torch.cuda.synchronize()
    u64 = u.astype(np.float64)
    for lo, hi in SAMPLE_BOXES_2D:
        ref = oracle.run_region("box", 2, 2, w, dims, u64, 20, lo, hi)
        got = y[lo[0] + 2:hi[0] + 2, lo[1] + 2:hi[1] + 2].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= TOL["f32"], (lo, hi)
    plan.close()
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("shape,r", [("star", 2), ("box", 1)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("t", [1, 2])
def test_config_3d_512_sampled(torch, shape, r, dtype, t):
    dims = (512, 512, 512)
    w, u = _big_problem(shape, 3, r, dims, 3, dtype)
    plan = B.Plan(shape, 3, r, w, dtype, dims, t)
    plan.set_option("path", "cuda_core")
    x = torch.from_numpy(np.array(u)).cuda()
    y = torch.empty_like(x)
    plan.run(x, y, 50)
    torch.cuda.synchronize()
    u64 = u.astype(np.float64)
    for lo, hi in (((0, 0, 0), (2, 3, 4)), ((255, 100, 509), (257, 102, 512)), ((511, 511, 0), (512, 512, 3))):
        ref = oracle.run_region(shape, 3, r, w, dims, u64, 50, lo, hi)
        got = y[lo[0] + r:hi[0] + r, lo[1] + r:hi[1] + r, lo[2] + r:hi[2] + r].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= TOL[dtype], (lo, hi)
    plan.close()
    del x, y
    torch.cuda.empty_cache()
