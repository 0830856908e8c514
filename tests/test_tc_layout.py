"""Host-side check of the tensor-core formulation (no GPU): the Toeplitz
operands the library issues, multiplied with an explicit im2col of the input
in numpy, reproduce the oracle's fused sweep, and the sparsity factor S the
dispatcher reports is the measured non-zero fraction of the issued blocks."""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import build as gbuild
from paper_2603_00477_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def lib():
    gbuild.build()
    return B.load()


def _plan(shape, r, dtype, precision, dims=(40, 50)):
    w = inputs.weights(shape, 2, r, seed=31)
    p = B.Plan(shape, 2, r, w, dtype, dims, 1)
    if dtype == "f32":
        p.set_option("precision", precision)
    p.set_option("path", "tensor_core")
    return p, w


CASES = [("box", 1, 1, "f64", "native"), ("box", 3, 2, "f64", "native"), ("star", 2, 3, "f64", "native"),
         ("box", 2, 1, "f32", "tf32"), ("box", 2, 4, "f32", "tf32"), ("star", 1, 4, "f32", "tf32x3"),
         ("star", 3, 2, "f32", "bf16x3"), ("box", 1, 7, "f32", "bf16x3"), ("box", 6, 2, "f32", "tf32")]


@pytest.mark.parametrize("shape,r,t,dtype,prec", CASES)
def test_toeplitz_times_im2col_equals_fused_sweep(shape, r, t, dtype, prec):
    p, w = _plan(shape, r, dtype, prec)
    lay, lo, hi, Bop = B.stencil_plan_tc_layout(p.handle, t)
    R, n, ki, nkb = lay["R"], lay["n_tile"], lay["k_inst"], lay["nkb"]
    assert R == t * r and lay["kext"] == nkb * ki and lay["kext"] >= n + 2 * R
    dims = (30, 384)  # a multiple of every MMA N the layouts use (8, 16, 32, 128)
    rng = np.random.default_rng(3)
    u = rng.uniform(0, 1, size=(dims[0] + 2 * R, dims[1] + 2 * R + lay["kext"]))
    # im2col: window of output columns x0..x0+n-1 of row y for line a is
    # u[y + a][x0 - R + k], k < kext (grid with a halo of width R)
    out = np.zeros(dims)
    for a in range(2 * R + 1):
        for x0 in range(0, dims[1], n):
            A = np.stack([u[a + y, x0: x0 + lay["kext"]] for y in range(dims[0])])  # (rows, kext)
            for kb in range(lo[a], hi[a] + 1):
                out[:, x0:x0 + n] += A[:, kb * ki:(kb + 1) * ki] @ Bop[a, kb]
    # oracle: one sweep of the composite kernel on a grid whose halo is R wide
    wt = oracle.compose(shape, 2, r, w, t)
    field = np.ascontiguousarray(u[:, :dims[1] + 2 * R])
    ref = oracle.apply_dense(2, wt, R, dims, field, margin=0)
    np.testing.assert_allclose(out, ref[R:R + dims[0], R:R + dims[1]], rtol=1e-13, atol=1e-13)
    # blocks that are not issued hold only zeros
    for a in range(2 * R + 1):
        for kb in range(nkb):
            if not (lo[a] <= kb <= hi[a]):
                assert not Bop[a, kb].any()
    # S = non-zeros / issued entries of the issued blocks (per output column)
    nnz = sum(np.count_nonzero(Bop[a, kb]) for a in range(2 * R + 1) for kb in range(lo[a], hi[a] + 1))
    issued = sum((hi[a] - lo[a] + 1) * ki * n for a in range(2 * R + 1))
    assert lay["sparsity"] == pytest.approx(nnz / issued)
    p.close()


@pytest.mark.parametrize("prec", ["tf32", "tf32x3"])
@pytest.mark.parametrize("t", [1, 2, 3, 4])
def test_sparsity_tf32_box2d2r(prec, t):
    """Box lines are all 2R+1 wide: S = (2R+1) / roundup(N + 2R, 8) for the
    MMA width N the kernel uses (32 when its operands fit, else 16 or 8)."""
    p, _ = _plan("box", 2, "f32", prec)
    lay = B.stencil_plan_tc_layout(p.handle, t, with_B=False)[0]
    R = 2 * t
    n = lay["n_tile"]
    assert n in (8, 16, 32)
    assert lay["sparsity"] == pytest.approx((2 * R + 1) / (-(-(n + 2 * R) // 8) * 8))
    if prec == "tf32":
        assert n == 32  # single-operand TF32 fits N = 32 up to R = 8
    p.close()


@pytest.mark.parametrize("t,S", [(1, 7 / 16), (2, 13 / 20), (3, 19 / 28), (4, 25 / 32)])
def test_sparsity_fp64_box2d3r(t, S):
    """FP64 MMA m8n8k4: S = (2R+1) / roundup(8 + 2R, 4)."""
    p, _ = _plan("box", 3, "f64", "native")
    assert B.stencil_plan_tc_layout(p.handle, t, with_B=False)[0]["sparsity"] == pytest.approx(S)
    p.close()


def test_plan_info_reports_layout_sparsity_and_alpha():
    from oracle import model
    p, _ = _plan("box", 2, "f32", "tf32", dims=(1000, 1000))
    p.set_option("t", 3)
    info = p.info()
    S = B.stencil_plan_tc_layout(p.handle, 3, with_B=False)[0]["sparsity"]
    assert info["path"] == B.PATH_TENSOR_CORE and info["t"] == 3
    assert info["sparsity"] == pytest.approx(S) and S == pytest.approx(13 / 48)
    assert info["alpha"] == pytest.approx(model.alpha("box", 2, 2, 3))
    assert info["intensity"] == pytest.approx(model.I_tc("box", 2, 2, 3, 4, S))
    p.close()


def test_layout_rejects_unsupported():
    p, _ = _plan("box", 3, "f64", "native")
    with pytest.raises(B.StencilError) as e:
        B.stencil_plan_tc_layout(p.handle, 5)  # R = 15 > 12
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    p.close()


@pytest.mark.parametrize("shape,r,t,dtype,prec", CASES + [("star", 2, 4, "f32", "tf32"), ("box", 3, 4, "f32", "tf32"),
                                                          ("star", 6, 2, "f32", "tf32x3")])
def test_tolerance_mma_count_is_the_band_count(shape, r, t, dtype, prec):
    """The MMA count the tensor-core tolerances use (tests/tc_bounds.py) comes
    from the band geometry alone, and the library's layout issues exactly it:
    a kernel issuing extra MMAs cannot loosen its own tolerance.  Pinned
    against S: Box-2D2R TF32 with N = 32, K = 8 issues 5 blocks of 8 per
    line at t = 1 (S = 5/40) and 6 at t = 4 (S = 17/48)."""
    from tc_bounds import dense_mma_per_output, line_half
    p, _ = _plan(shape, r, dtype, prec)
    lay, lo, hi, _ = B.stencil_plan_tc_layout(p.handle, t, with_B=False)
    n = dense_mma_per_output(shape, r, t, lay["n_tile"], lay["k_inst"])
    assert sum(max(0, h - l + 1) for l, h in zip(lo, hi)) == n
    useful = sum(2 * line_half(shape, r, t, a) + 1 for a in range(-t * r, t * r + 1) if line_half(shape, r, t, a) >= 0)
    assert lay["sparsity"] == pytest.approx(useful / (n * lay["k_inst"]))
    p.close()
    assert dense_mma_per_output("box", 2, 1, 32, 8) == 5 * 5
    assert dense_mma_per_output("box", 2, 4, 32, 8) == 17 * 6


@pytest.mark.parametrize("shape,r,t", [("box", 2, 1), ("box", 2, 2), ("box", 2, 3), ("box", 2, 4), ("star", 2, 3),
                                       ("star", 6, 2), ("box", 3, 4), ("box", 7, 1), ("box", 1, 3)])
def test_sparse_tolerance_count_bounds_the_layout(shape, r, t):
    """The sparse tolerance's instruction count (ceil(nc/2) per non-empty line,
    nc = ceil((16 + 2R)/4) chunks: every chunk paired with a dummy at worst)
    is an upper bound of what the layout issues.  For Box-2D2R the layout
    issues what the pinned S gives: t = 1..3 two instructions per line
    (25/160, 81/288, 169/416), t = 4 three (289/816)."""
    from tc_bounds import sparse_mma_bound
    w = inputs.weights(shape, 2, r, seed=31)
    p = B.Plan(shape, 2, r, w, "f32", (40, 50), t)
    mask = B.stencil_plan_sptc_layout(p.handle, t)[3]
    p.close()
    issued = int(sum(bin(int(m)).count("1") for m in mask))
    assert issued <= sparse_mma_bound(shape, r, t)
    assert [sparse_mma_bound("box", 2, tt) for tt in (1, 2, 3, 4)] == [5 * 3, 9 * 3, 13 * 4, 17 * 4]
    if (shape, r) == ("box", 2):
        useful = {1: 25, 2: 81, 3: 169, 4: 289}[t]
        S = {1: 25 / 160, 2: 81 / 288, 3: 169 / 416, 4: 289 / 816}[t]
        assert issued == round(useful / S / 16)
