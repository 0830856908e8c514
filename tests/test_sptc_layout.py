"""Host-side check of the 2:4-structured sparse formulation (paper Sec. 4.3;
no GPU): the compressed Toeplitz operands the sparse kernel issues, expanded
through the exported K permutation and selectors, are exactly the Toeplitz
blocks of the oracle's composite kernel w^(t) (to TF32 rounding of each
weight); every pair of logical K keeps at most one band entry (the 1:2 rule of
TF32 sparsity); their product with an im2col of the input reproduces the
oracle's fused sweep; and S is the useful fraction of the logical MACs
issued."""
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


def _plan(shape, r, t):
    w = inputs.weights(shape, 2, r, seed=41 + r)
    p = B.Plan(shape, 2, r, w, "f32", (40, 50), 1)
    p.set_option("precision", "tf32")
    return p, w


def _expand(R, cf, cs, vals, sel, a, s):
    """Logical 16 x (window) Toeplitz of line a from instruction s: dict
    (m, column) -> value, and the set of columns each logical pair maps to."""
    T = {}
    for m in range(16):
        for p in range(8):
            cp, i = 2 * s + (p & 1), p >> 1
            chunk = (cs if sel[a, s, m, p] else cf)[cp]
            v = float(vals[a, s, m, p])
            if chunk < 0:
                assert v == 0.0  # a dummy chunk carries no weight
                continue
            if v != 0.0:
                col = 4 * chunk + i
                assert (m, col) not in T
                T[(m, col)] = v
    return T


CASES = [("box", 1, 1), ("box", 2, 1), ("box", 2, 2), ("box", 2, 4), ("box", 3, 4), ("box", 1, 7),
         ("star", 2, 3), ("star", 1, 4), ("box", 6, 2), ("star", 4, 3), ("box", 4, 3)]


@pytest.mark.parametrize("shape,r,t", CASES)
def test_sparse_operands_are_the_composite_toeplitz(shape, r, t):
    p, w = _plan(shape, r, t)
    lay, cf, cs, mask, vals, sel = B.stencil_plan_sptc_layout(p.handle, t)
    R, ns = lay["R"], lay["ns"]
    assert R == t * r and lay["nc"] == -(-(16 + 2 * R) // 4)
    # pairs: members at least 2R+1 columns apart -> no row's band holds both
    for f, s2 in zip(cf, cs):
        if f >= 0 and s2 >= 0:
            assert 4 * abs(int(s2) - int(f)) >= 2 * R + 1
    # every window chunk appears in exactly one pair
    chunks = sorted(int(c) for c in list(cf) + list(cs) if c >= 0)
    assert chunks == list(range(lay["nc"]))
    wt = oracle.compose(shape, 2, r, w, t)  # (2R+1) x (2R+1), FP64
    lines = 2 * R + 1
    issued = 0
    for a in range(lines):
        T = {}
        for s in range(ns):
            Ts = _expand(R, cf, cs, vals, sel, a, s)
            if not (mask[a] >> s) & 1:
                assert not Ts  # skipped instructions hold no weight
                continue
            issued += 16
            for k, v in Ts.items():
                assert k not in T
                T[k] = v
        expect = {(m, m + b): wt[a, b] for m in range(16) for b in range(2 * R + 1) if wt[a, b] != 0.0}
        assert set(T) == set(expect)
        for k, v in T.items():
            assert abs(v - expect[k]) <= 2.0 ** -11 * abs(expect[k])  # TF32 keeps 11 significant bits
    useful = np.count_nonzero(wt)
    assert lay["sparsity"] == pytest.approx(useful / issued)
    p.close()


@pytest.mark.parametrize("shape,r,t", [("box", 2, 1), ("box", 2, 3), ("star", 3, 2), ("box", 1, 9)])
def test_sparse_product_equals_fused_sweep(shape, r, t):
    """Sum over lines and instructions of A (expanded) x im2col(input) equals
    one sweep of the composite kernel with the TF32-rounded weights."""
    p, w = _plan(shape, r, t)
    lay, cf, cs, mask, vals, sel = B.stencil_plan_sptc_layout(p.handle, t)
    R, ns, nc = lay["R"], lay["ns"], lay["nc"]
    dims = (24, 48)  # 3 strips of 16 output columns
    rng = np.random.default_rng(5)
    u = rng.uniform(0, 1, size=(dims[0] + 2 * R, dims[1] + 4 * nc))
    out = np.zeros(dims)
    wr = np.zeros((2 * R + 1, 2 * R + 1))
    for a in range(2 * R + 1):
        for s in range(ns):
            if not (mask[a] >> s) & 1:
                continue
            for (m, col), v in _expand(R, cf, cs, vals, sel, a, s).items():
                wr[a, col - m] = v
                for x0 in range(0, dims[1], 16):
                    out[:, x0 + m] += v * u[a:a + dims[0], x0 + col]
    field = np.ascontiguousarray(u[:, :dims[1] + 2 * R])
    ref = oracle.apply_dense(2, wr, R, dims, field, margin=0)
    np.testing.assert_allclose(out, ref[R:R + dims[0], R:R + dims[1]], rtol=1e-13, atol=1e-13)
    # and the rounded composite is the oracle's composite to TF32 precision
    wt = oracle.compose(shape, 2, r, w, t)
    assert np.max(np.abs(wr - wt)) <= 2.0 ** -11 * np.max(np.abs(wt))
    p.close()


@pytest.mark.parametrize("t,S", [(1, 25 / 160), (2, 81 / 288), (3, 169 / 416), (4, 289 / 816)])
def test_sparse_S_box2d2r(t, S):
    """Box-2D2R: useful (2R+1)^2 per output over 16 logical K per issued
    instruction; R <= 7 needs two instructions per line, R = 8 three."""
    p, _ = _plan("box", 2, t)
    lay = B.stencil_plan_sptc_layout(p.handle, t)[0]
    assert lay["sparsity"] == pytest.approx(S)
    p.close()


def test_sparse_plan_info_and_rejects():
    p, _ = _plan("box", 2, 1)
    p.set_option("path", "sparse_tensor_core")
    p.set_option("t", 2)
    info = p.info()
    assert info["path"] == B.PATH_SPARSE_TENSOR_CORE and info["t"] == 2
    assert info["sparsity"] == pytest.approx(81 / 288)
    p.close()
    w = inputs.weights("box", 2, 3, seed=1)
    q = B.Plan("box", 2, 3, w, "f64", (40, 40), 1)
    with pytest.raises(B.StencilError) as e:
        q.set_option("path", "sparse_tensor_core")  # no FP64 sparse MMA
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    with pytest.raises(B.StencilError) as e:
        B.stencil_plan_sptc_layout(q.handle, 1)
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    q.close()
