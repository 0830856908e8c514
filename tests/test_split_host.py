"""Host-side checks of FP64 by exact splitting (precision "ozaki"; no GPU).

1. The digit width the library picks is the one the exactness condition
   fixes: re-derived here from the oracle's composite kernel w^(t) with a
   digit cut written in Python integers, the smallest S in {6, 7} (b = 9, 8
   bits per digit, S b - 1 >= 53 fixed-point bits) for which every product
   level L = i + j < S has 2^(b-1) * sum_{j<=L} sum_taps |b_j| < 2^24.
2. The scheme itself (the Ozaki-type splitting: balanced digits, exact
   per-level integer sums, levels i + j >= S dropped, one rounding), emulated
   in Python integers on a small grid, reproduces the oracle's FP64 sweep to
   a few units of 2^-53 normwise; dropping one more level (L = S - 1) or one
   digit of the field breaks that, so the test pins how many levels and
   digits FP64 accuracy needs.
"""
import math

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


def balanced_digits(V: int, b: int, S: int) -> list:
    """V = sum_i d_i 2^(b(S-1-i)), |d_i| <= 2^(b-1) (top digit first)."""
    out = []
    for _ in range(S - 1):
        d = V % (1 << b)
        if d >= 1 << (b - 1):
            d -= 1 << b
        out.append(d)
        V = (V - d) >> b
    out.append(V)
    return out[::-1]


def fixed_point(x: float, E: int, NB: int) -> int:
    """round(x * 2^(NB - E)) with |x| < 2^E, exactly (Python integers)."""
    m, e = math.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    num = int(m * (1 << 53))
    sh = e - 53 + NB - E
    if sh >= 0:
        return num << sh
    q, rem = divmod(abs(num), 1 << -sh)
    if 2 * rem >= 1 << -sh:
        q += 1
    return q if num >= 0 else -q


def expected_slices(wt: np.ndarray):
    wmax = float(np.max(np.abs(wt)))
    Ew = math.frexp(wmax)[1]
    for S, b in ((6, 9), (7, 8)):
        NB = S * b - 1
        digs = [balanced_digits(fixed_point(float(x), Ew, NB), b, S) for x in wt.ravel()]
        cum = 0
        ok = True
        for L in range(S):
            cum += sum(abs(d[L]) for d in digs)
            if (cum << (b - 1)) >= 1 << 24:
                ok = False
        if ok:
            return S
    return None


CASES = [("box", 3, 1, 2), ("box", 1, 3, 5), ("box", 2, 3, 7), ("star", 2, 2, 11), ("star", 4, 2, 13),
         ("box", 1, 4, 17), ("star", 1, 4, 19)]


@pytest.mark.parametrize("shape,r,t,seed", CASES)
def test_digit_width_is_the_exactness_condition(shape, r, t, seed):
    w = inputs.weights(shape, 2, r, seed)
    wt = oracle.compose(shape, 2, r, w, t)
    S = expected_slices(wt)
    p = B.Plan(shape, 2, r, w, "f64", (300, 300), t)
    # shared memory holds the 7-digit tiles (S = 7) up to a fused radius of 6
    if S is None or (S == 7 and t * r > 6):
        with pytest.raises(B.StencilError):
            p.set_option("precision", "ozaki")
            p.set_option("path", "tensor_core")
        return
    p.set_option("precision", "ozaki")
    p.set_option("path", "tensor_core")
    info = p.info()
    p.close()
    assert info["beta"] == S * (S + 1) / 2
    assert info["precision"] == B.PREC_OZAKI


def test_large_weight_digits_take_the_narrower_digits():
    """Weights whose 9-bit digits are all near +-255 break the b = 9 bound at
    level 5 (6 * 49 * 255 * 256 > 2^24); 8-bit digits (S = 7) qualify."""
    Ew, NB = 0, 53
    rng = np.random.default_rng(3)
    w = []
    for _ in range(49):
        digs = [int(rng.choice([-1, 1]) * rng.integers(240, 256)) for _ in range(6)]
        digs[0] = abs(digs[0])
        V = sum(d << (9 * (5 - i)) for i, d in enumerate(digs))
        w.append(math.ldexp(V, Ew - NB))
    w = np.array(w)
    assert expected_slices(w) == 7
    p = B.Plan("box", 2, 3, w, "f64", (200, 200), 1)
    p.set_option("precision", "ozaki")
    p.set_option("path", "tensor_core")
    assert p.info()["beta"] == 28
    p.close()


def test_fp64_plans_pick_the_split_form_only_when_asked():
    """precision native (the default) keeps FP64 arithmetic; ozaki and any
    may take the split form; FP32 grids refuse ozaki."""
    w = inputs.weights("box", 2, 3, 2)
    p = B.Plan("box", 2, 3, w, "f64", (4096, 4096), 0)
    assert p.info()["precision"] == B.PREC_NATIVE
    p.set_option("precision", "ozaki")
    assert p.info()["precision"] == B.PREC_OZAKI and p.info()["path"] == B.PATH_TENSOR_CORE
    p.close()
    q = B.Plan("box", 2, 2, inputs.weights("box", 2, 2, 4), "f32", (256, 256), 0)
    with pytest.raises(B.StencilError):
        q.set_option("precision", "ozaki")
    q.close()


def _emulated_sweep(u, wt, R, S, b, levels):
    """One sweep of the split scheme on the whole stored grid u (one tile):
    fixed point of u and w^(t), balanced digits, exact level sums for
    L < levels, recombination, one rounding."""
    NB = S * b - 1
    Eu = math.frexp(float(np.max(np.abs(u))))[1]
    Ew = math.frexp(float(np.max(np.abs(wt))))[1]
    ud = np.array([[balanced_digits(fixed_point(float(x), Eu, NB), b, S) for x in row] for row in u], dtype=object)
    wd = np.array([[balanced_digits(fixed_point(float(x), Ew, NB), b, S) for x in row] for row in wt], dtype=object)
    ny, nx = u.shape[0] - 2 * R, u.shape[1] - 2 * R
    out = np.zeros((ny, nx))
    for y in range(ny):
        for x in range(nx):
            tot = 0
            for L in range(levels):
                sL = 0
                for i in range(L + 1):
                    j = L - i
                    if i >= S or j >= S:
                        continue
                    for a in range(2 * R + 1):
                        for c in range(2 * R + 1):
                            sL += ud[y + a, x + c][i] * wd[a, c][j]
                assert abs(sL) < 1 << 24
                tot += sL << (b * (S - 1 - L))
            # tot * 2^(b(S-1)) * 2^(Eu + Ew - 2 NB), rounded once
            out[y, x] = math.ldexp(float(tot), b * (S - 1) + Eu + Ew - 2 * NB)
    return out


def test_split_scheme_emulation_meets_fp64():
    R, dims = 3, (10, 12)
    w, u = inputs.problem("box", 2, R, dims, seed=53, dtype=np.float64)
    wt = oracle.compose("box", 2, R, w, 1)
    ref = oracle.run("box", 2, R, w, dims, u, 1)[R:-R, R:-R]
    full = _emulated_sweep(u, wt, R, 6, 9, 6)
    assert oracle.rel_linf(full, ref) <= 4 * 2.0 ** -53
    # one level fewer (L <= 4): the level-5 products are ~2^-45 of the result
    fewer = _emulated_sweep(u, wt, R, 6, 9, 5)
    assert oracle.rel_linf(fewer, ref) > 16 * 2.0 ** -53
    # one digit fewer (S = 5, 44 bits): the cut of u alone costs ~2^-45
    short = _emulated_sweep(u, wt, R, 5, 9, 5)
    assert oracle.rel_linf(short, ref) > 16 * 2.0 ** -53
