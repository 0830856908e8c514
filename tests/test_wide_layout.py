"""Host checks of the wide FP16 tensor-core kernel's operand addressing (no GPU).

The wide kernel (precisions f16 / f16x3 where its operands fit) makes the
Toeplitz factor of line a the A operand: M = 128 output columns stored in
reverse order (row m' is output column 127 - m'), K = 16 nkb window columns
(window column k is input column x0 - R + k).  With that order
A_a[m'][k] = w^(t)[a][k + m' - 127], so each line keeps one strip of core
matrices (8 rows x 8 FP16, 128 bytes) and the MMA of K block kb reads core
matrix (m' group g, k chunk c) at strip index J = 2 kb + c + g (LBO = SBO =
128 bytes); the strips of consecutive lines are delta core matrices apart and
overlap where both are zero.

This test builds the strips the way the kernel does (zero everything, then
write each line's non-zero core matrices) and reads every issued (line, K
block) operand back through that address arithmetic: each must equal the
Toeplitz block of the oracle's composite kernel, the blocks a line skips must
be zero in the Toeplitz matrix, every read must stay inside the strips, and
the input tile's rows and chunk columns read by the B descriptors must lie
inside the staged tile.
"""
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


def geom(R, nr, split, nbuf=2):
    nkb = (128 + 2 * R + 15) // 16
    strip_len = 2 * nkb + 15
    delta = max(2 * nkb, (127 + 2 * R) // 8 + 1)
    hs = (nr + 2 * R) | 1
    strip_bytes = (2 * R * delta + strip_len) * 128
    in_bytes = 2 * nkb * hs * 16
    smem = 1024 + (strip_bytes + nbuf * in_bytes) * (2 if split else 1)
    return nkb, delta, hs, strip_bytes, smem


def half_width(shape, r, t, a):
    R = t * r
    if shape == "box":
        return R
    ca = -(-abs(a) // r)
    return -1 if ca > t else r * (t - ca)


CASES = [("box", 1, 1), ("box", 2, 1), ("box", 2, 4), ("star", 2, 3), ("box", 3, 3), ("star", 4, 2),
         ("box", 1, 9), ("star", 3, 4), ("box", 6, 2), ("star", 1, 12), ("box", 7, 1)]


@pytest.mark.parametrize("shape,r,t", CASES)
def test_strip_operands_are_the_toeplitz_blocks(shape, r, t):
    R = t * r
    lines = 2 * R + 1
    w = inputs.weights(shape, 2, r, 5)
    wt = oracle.compose(shape, 2, r, w, t)  # (2R+1) x (2R+1)
    nr = 256 if geom(R, 256, False)[4] <= 227 * 1024 else 128
    nkb, delta, hs, strip_bytes, smem = geom(R, nr, False)
    assert smem <= 227 * 1024
    # the strips as the kernel writes them (values in place of FP16 bits)
    mem = np.zeros(strip_bytes // 2)
    filled = np.zeros(strip_bytes // 2, dtype=int)
    for ai in range(lines):
        for J in range(15, (127 + 2 * R) // 8 + 1):
            for ii in range(8):
                for jj in range(8):
                    idx = 8 * J + ii + jj - 127
                    if 0 <= idx <= 2 * R:
                        off = (ai * delta + J) * 64 + ii * 8 + jj
                        assert filled[off] == 0, "two lines write the same strip element"
                        filled[off] = 1
                        mem[off] = wt[ai, idx]
    # every issued (line, K block): the descriptor's reads against the Toeplitz block
    mp = np.arange(128)[:, None]        # reversed output column m'
    kk = np.arange(16)[None, :]         # K within the block
    g, ii = mp // 8, mp % 8
    c, jj = kk // 8, kk % 8
    lay = B.Plan(shape, 2, r, w, "f32", (4096, 4096), t)
    lay.set_option("precision", "f16")
    lay.set_option("path", "tensor_core")
    info, lo, hi, _ = B.stencil_plan_tc_layout(lay.handle, t, with_B=False)
    lay.close()
    assert info["n_tile"] == 128 and info["k_inst"] == 16
    for ai in range(lines):
        h = half_width(shape, r, t, ai - R)
        row = wt[ai]
        for kb in range(nkb):
            kabs = 16 * kb + kk
            tap = kabs + mp - 127  # weight index of (output column 127 - m', window column kabs)
            want = np.where((tap >= 0) & (tap <= 2 * R), row[np.clip(tap, 0, 2 * R)], 0.0)
            issued = lo[ai] <= kb <= hi[ai]
            if not issued:
                assert not want.any(), (ai, kb)
                continue
            addr = (ai * delta + 2 * kb + c + g) * 64 + ii * 8 + jj
            assert addr.min() >= 0 and addr.max() < mem.size
            np.testing.assert_array_equal(mem[addr], want)
        if h < 0:
            assert lo[ai] > hi[ai]
    # B operand: line ai reads staged rows ai .. ai + nr - 1 and chunk columns 2 kb, 2 kb + 1
    assert 2 * R + nr - 1 < hs
    assert max(hi) * 2 + 1 < 2 * nkb


def test_wide_tiles_fit():
    """N = 256 output rows with two operand buffers up to R = 9 (f16), 128
    above; the hi + lo forms (f16x3, bf16x3) at N = 128 with two buffers up to
    R = 6 and with one buffer up to R = 12, so every fused radius the
    tensor-core path takes (t r <= 12) has a wide tile.  The plan reports
    the wide geometry (128 output columns a tile) for all of them."""
    order = ((256, 2), (128, 2), (128, 1))
    for R in range(1, 13):
        f16 = next((c for c in order if geom(R, c[0], False, c[1])[4] <= 227 * 1024), None)
        hl = next((c for c in order if geom(R, c[0], True, c[1])[4] <= 227 * 1024), None)
        assert f16 == ((256, 2) if R <= 9 else (128, 2)), R
        assert hl == ((128, 2) if R <= 6 else (128, 1)), R
        # TMEM: two accumulators of N FP32 columns
        assert 2 * f16[0] <= 512 and 2 * hl[0] <= 512
    w = inputs.weights("box", 2, 1, 3)
    for t, prec in ((4, "f16"), (7, "f16x3"), (11, "f16x3"), (12, "f16"), (12, "bf16x3")):
        p = B.Plan("box", 2, 1, w, "f32", (2048, 2048), t)
        p.set_option("precision", prec)
        p.set_option("path", "tensor_core")
        info = B.stencil_plan_tc_layout(p.handle, t, with_B=False)[0]
        p.close()
        assert info["n_tile"] == 128, (t, prec)


def geom3(R, nlines, nr):
    nkb = (128 + 2 * R + 15) // 16
    delta = max(2 * nkb, (127 + 2 * R) // 8 + 1)
    hs = (nr + 2 * R) | 1
    strip_bytes = ((nlines - 1) * delta + 2 * nkb + 15) * 128
    return 1024 + 2 * strip_bytes + (2 * R + 2) * 2 * nkb * hs * 16


@pytest.mark.parametrize("shape,r,want_nr", [("box", 1, 128), ("star", 1, 128), ("star", 2, 64), ("box", 2, 32),
                                             ("star", 3, 64)])
def test_wide3_tiles_and_sparsity(shape, r, want_nr):
    """The 3-D FP16 kernel: two strip sets of the (dz, dy) lines and a ring of
    2r + 2 plane tiles in 227 KB decide the rows per tile; the plan reports
    that tile and S = useful / issued MACs, each line issuing the K blocks of
    its 128 + 2r window that hold a non-zero column."""
    lines = [r] * (2 * r + 1) ** 2 if shape == "box" else [r] + [0] * (4 * r)
    nr = next(n for n in (128, 64, 32) if geom3(r, len(lines), n) <= 227 * 1024)
    assert nr == want_nr
    nkb = -(-(128 + 2 * r) // 16)
    issued = sum((min(nkb - 1, (r + h + 127) // 16) - (r - h) // 16 + 1) * 16 for h in lines)
    useful = sum(2 * h + 1 for h in lines)
    w = inputs.weights(shape, 3, r, 1)
    p = B.Plan(shape, 3, r, w, "f32", (64, 64, 64), 1)
    p.set_option("precision", "f16")
    p.set_option("path", "tensor_core")
    info = p.info()
    p.close()
    assert info["tile"] == [1, nr, 128]
    assert info["sparsity"] == pytest.approx(useful / issued, rel=1e-12)


def test_wide3_only_fp16_one_step():
    """3-D grids take the tensor cores only as FP32 in the FP16 form at t = 1."""
    w = inputs.weights("box", 3, 1, 1)
    for dtype, prec, t in (("f64", None, 1), ("f32", "tf32", 1), ("f32", "f16", 2)):
        p = B.Plan("box", 3, 1, w, dtype, (32, 32, 32), t)
        with pytest.raises(B.StencilError):
            if prec:
                p.set_option("precision", prec)
            p.set_option("path", "tensor_core")
            p.info()
        p.close()
