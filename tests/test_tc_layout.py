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
    dims = (30, 96)  # a multiple of every MMA N the layouts use (8, 16, 32)
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
