"""Pins of the CPU oracle against things other than itself.

Each test ties the oracle (oracle/oracle.c) to a library routine, a closed
form, an exact special case or brute force, chosen so that a plausible slip
(a transposed offset, a wrong sign, a dropped term, a halo that moves, a
reversed convolution) fails at least one of them.
"""
import itertools

import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

import oracle
from oracle import model
from paper_2603_00477_gb300 import inputs

CASES_2D = [("box", 1, (7, 9)), ("star", 1, (8, 5)), ("box", 2, (6, 11)), ("star", 3, (9, 7)),
            ("box", 3, (2, 3)), ("star", 2, (1, 1)), ("box", 1, (1, 6))]
CASES_3D = [("box", 1, (4, 5, 3)), ("star", 2, (3, 4, 5)), ("star", 1, (1, 2, 3)), ("box", 2, (2, 2, 2))]


def _problem(shape, d, r, dims, seed, nonsym=True):
    w, u = inputs.problem(shape, d, r, dims, seed)
    # a non-zero halo exercises the fixed boundary as well
    rng = np.random.default_rng(seed)
    halo = rng.uniform(-1.0, 1.0, size=u.shape)
    inner = tuple(slice(r, r + n) for n in dims)
    halo[inner] = u[inner]
    return w, halo


def _dense_kernel(shape, d, r, w):
    """Scatter the K weights into a dense (2r+1)^d box by their offsets."""
    side = 2 * r + 1
    dense = np.zeros((side,) * d)
    for wk, o in zip(w, oracle.offsets(shape, d, r)):
        dense[tuple(int(c) + r for c in o)] = wk
    return dense


# --- offsets and K -----------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r", [1, 2, 3])
def test_offsets_order_and_count(d, r):
    box = list(itertools.product(range(-r, r + 1), repeat=d))  # lexicographic, first axis outermost
    star = [o for o in box if sum(c != 0 for c in o) <= 1]
    assert [tuple(o) for o in oracle.offsets("box", d, r)] == box
    assert [tuple(o) for o in oracle.offsets("star", d, r)] == star
    assert len(box) == (2 * r + 1) ** d == model.K_points("box", d, r)
    assert len(star) == 2 * d * r + 1 == model.K_points("star", d, r)


# --- one step against scipy.ndimage.correlate (a library routine) -------------------

@pytest.mark.parametrize("shape,r,dims", CASES_2D)
def test_step_matches_scipy_correlate_2d(shape, r, dims):
    w, u = _problem(shape, 2, r, dims, seed=11)
    ref = scipy.ndimage.correlate(u, _dense_kernel(shape, 2, r, w), mode="constant", cval=0.0)
    got = oracle.step(shape, 2, r, w, dims, u)
    inner = tuple(slice(r, r + n) for n in dims)
    np.testing.assert_allclose(got[inner], ref[inner], rtol=1e-13, atol=1e-13)
    halo_mask = np.ones(u.shape, bool)
    halo_mask[inner] = False
    assert np.array_equal(got[halo_mask], u[halo_mask])


@pytest.mark.parametrize("shape,r,dims", CASES_3D)
def test_step_matches_scipy_correlate_3d(shape, r, dims):
    w, u = _problem(shape, 3, r, dims, seed=12)
    ref = scipy.ndimage.correlate(u, _dense_kernel(shape, 3, r, w), mode="constant", cval=0.0)
    got = oracle.step(shape, 3, r, w, dims, u)
    inner = tuple(slice(r, r + n) for n in dims)
    np.testing.assert_allclose(got[inner], ref[inner], rtol=1e-13, atol=1e-13)


def test_step_is_correlation_not_convolution():
    """A one-hot weight at offset (0, +1) must read the right neighbour."""
    dims = (4, 5)
    u = np.zeros((6, 7))
    u[1:5, 1:6] = np.arange(20, dtype=float).reshape(4, 5)
    w = np.zeros(9)
    w[5] = 1.0  # offsets order: index 5 is (0, +1)
    assert tuple(oracle.offsets("box", 2, 1)[5]) == (0, 1)
    got = oracle.step("box", 2, 1, w, dims, u)
    assert np.array_equal(got[1:5, 1:6], u[1:5, 2:7])


# --- many steps against an explicitly assembled stencil matrix ---------------------

def _assemble(shape, d, r, w, dims):
    """Affine map u_int -> A u_int + b on the interior, assembled entry by entry."""
    dims = tuple(dims)
    n = int(np.prod(dims))
    A = np.zeros((n + 1, n + 1))
    A[n, n] = 1.0
    interior = list(itertools.product(*[range(k) for k in dims]))
    index = {p: i for i, p in enumerate(interior)}
    return A, index, interior


@pytest.mark.parametrize("shape,d,r,dims,steps", [
    ("box", 2, 1, (5, 6), 7), ("star", 2, 2, (6, 4), 5), ("box", 2, 3, (3, 2), 4),
    ("star", 2, 1, (1, 1), 3), ("box", 3, 1, (3, 4, 2), 4), ("star", 3, 2, (2, 3, 3), 3)])
def test_run_matches_matrix_power(shape, d, r, dims, steps):
    w, u = _problem(shape, d, r, dims, seed=13)
    A, index, interior = _assemble(shape, d, r, w, dims)
    n = len(interior)
    offs = oracle.offsets(shape, d, r)
    for p in interior:
        row = index[p]
        for wk, o in zip(w, offs):
            q = tuple(p[i] + int(o[i]) for i in range(d))
            if all(0 <= q[i] < dims[i] for i in range(d)):
                A[row, index[q]] += wk
            else:  # a fixed halo cell: constant term
                A[row, n] += wk * u[tuple(q[i] + r for i in range(d))]
    x = np.ones(n + 1)
    x[:n] = [u[tuple(c + r for c in p)] for p in interior]
    ref = np.linalg.matrix_power(A, steps) @ x
    got = oracle.run(shape, d, r, w, dims, u, steps)
    got_int = np.array([got[tuple(c + r for c in p)] for p in interior])
    np.testing.assert_allclose(got_int, ref[:n], rtol=1e-12, atol=1e-12)


# --- composite kernel and fusion ---------------------------------------------------

@pytest.mark.parametrize("shape,d,r,t", [("box", 2, 1, 3), ("star", 2, 2, 2), ("star", 3, 1, 3),
                                         ("box", 3, 1, 2), ("box", 1, 2, 4), ("star", 2, 1, 4)])
def test_compose_matches_scipy_convolve(shape, d, r, t):
    w = inputs.weights(shape, d, r, seed=21)
    dense = _dense_kernel(shape, d, r, w)
    ref = np.ones((1,) * d)
    for _ in range(t):
        ref = scipy.signal.convolve(ref, dense, mode="full", method="direct")
    got = oracle.compose(shape, d, r, w, t)
    assert got.shape == ref.shape
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("shape,d,r,t", [("box", 2, 1, 1), ("box", 2, 1, 3), ("box", 2, 3, 2),
                                         ("star", 2, 1, 5), ("star", 2, 2, 3), ("star", 3, 2, 2),
                                         ("box", 3, 1, 3), ("star", 3, 1, 4)])
def test_compose_support_and_sum(shape, d, r, t):
    w = inputs.weights(shape, d, r, seed=22) * 1.7  # taps sum to 1.7
    wt = oracle.compose(shape, d, r, w, t)
    # sum of the taps of w^(t) is (sum w)^t
    assert abs(wt.sum() - 1.7 ** t) < 1e-12 * 1.7 ** t
    # support = Minkowski sum of t offset sets, enumerated by brute force
    offs = {tuple(o) for o in oracle.offsets(shape, d, r)}
    support = {(0,) * d}
    for _ in range(t):
        support = {tuple(a + b for a, b in zip(s, o)) for s in support for o in offs}
    assert int(np.count_nonzero(wt)) == len(support) == model.K_fused(shape, d, r, t)


def test_fusion_example_box2d1r_t3():
    """Sec. 2.2.3: Box-2D1R fused over 3 steps covers 7x7 = 49 points versus
    3 x 9 = 27 stepwise, i.e. 22 redundant multiply-adds per output."""
    w = inputs.weights("box", 2, 1, seed=3)
    wt = oracle.compose("box", 2, 1, w, 3)
    assert wt.shape == (7, 7) and np.count_nonzero(wt) == 49
    assert model.K_fused("box", 2, 1, 3) - 3 * model.K_points("box", 2, 1) == 22


@pytest.mark.parametrize("shape,d,r,t,dims", [("box", 2, 1, 3, (17, 19)), ("star", 2, 2, 2, (15, 12)),
                                              ("box", 2, 3, 4, (30, 31)), ("star", 3, 1, 3, (9, 10, 8)),
                                              ("box", 3, 1, 2, (7, 8, 9))])
def test_fused_sweep_equals_t_steps_on_shrunk_interior(shape, d, r, t, dims):
    """Closed form: t stepwise sweeps = one sweep of w^(t) wherever the fused
    neighbourhood stays clear of the fixed halo (distance >= (t-1) r)."""
    w, u = _problem(shape, d, r, dims, seed=14)
    stepwise = oracle.run(shape, d, r, w, dims, u, t)
    wt = oracle.compose(shape, d, r, w, t)
    m = (t - 1) * r
    fused = oracle.apply_dense(d, wt, r, dims, u, margin=m)
    region = tuple(slice(r + m, r + n - m) for n in dims)
    assert stepwise[region].size > 0
    np.testing.assert_allclose(fused[region], stepwise[region], rtol=1e-13, atol=1e-13)
    # next to the halo the fused form differs: the halo is re-imposed after
    # every step, which one fused sweep over a wider halo cannot reproduce
    if t > 1:
        padded = np.pad(u, (t - 1) * r)
        fused_all = oracle.apply_dense(d, wt, t * r, dims, padded, margin=0)
        edge = tuple(slice(t * r, t * r + 1) for _ in dims)
        sedge = tuple(slice(r, r + 1) for _ in dims)
        assert abs(fused_all[edge].item() - stepwise[sedge].item()) > 1e-6


# --- invariants and exact special cases --------------------------------------------

@pytest.mark.parametrize("shape,d,r,dims,steps", [("box", 2, 2, (20, 23), 9), ("star", 3, 1, (8, 9, 7), 6),
                                                  ("star", 2, 3, (13, 13), 12)])
def test_constant_field_preserved(shape, d, r, dims, steps):
    w = inputs.weights(shape, d, r, seed=31)
    c = 0.8125
    u = np.full(tuple(n + 2 * r for n in dims), c)
    got = oracle.run(shape, d, r, w, dims, u, steps)
    K = len(w)
    assert np.max(np.abs(got - c)) <= 4 * K * steps * np.finfo(float).eps
    # zero halo: points farther than steps*r from the boundary keep the constant
    u0 = np.zeros_like(u)
    inner = tuple(slice(r, r + n) for n in dims)
    u0[inner] = c
    got0 = oracle.run(shape, d, r, w, dims, u0, steps)
    far = tuple(slice(r + steps * r, r + n - steps * r) for n in dims)
    if got0[far].size:
        assert np.max(np.abs(got0[far] - c)) <= 4 * K * steps * np.finfo(float).eps
    near = tuple(slice(r, r + 1) for _ in dims)
    assert np.all(got0[near] < c)  # the zero halo pulls the edge down


@pytest.mark.parametrize("shape,d,r", [("box", 2, 2), ("star", 3, 2), ("star", 2, 1)])
def test_one_hot_weight_is_exact_shift(shape, d, r):
    offs = oracle.offsets(shape, d, r)
    k = len(offs) - 1  # last offset: +r along the last axis
    w = np.zeros(len(offs))
    w[k] = 1.0
    dims = (9,) * d if d == 2 else (5, 6, 9)
    _, u = _problem(shape, d, r, dims, seed=32)
    steps = 2
    got = oracle.run(shape, d, r, w, dims, u, steps)
    shift = steps * np.asarray(offs[k])
    region = tuple(slice(r, r + n - steps * r) for n in dims)
    src = tuple(slice(r + int(s), r + n - steps * r + int(s)) for n, s in zip(dims, shift))
    assert np.array_equal(got[region], u[src])


def test_identity_weight_is_bitwise_identity():
    w = np.zeros(9)
    w[4] = 1.0
    _, u = _problem("box", 2, 1, (10, 7), seed=33)
    assert np.array_equal(oracle.run("box", 2, 1, w, (10, 7), u, 5), u)


@pytest.mark.parametrize("shape,d,r,dims", [("box", 2, 3, (12, 17)), ("star", 3, 2, (6, 7, 5))])
def test_dyadic_weights_integer_field_exact(shape, d, r, dims):
    """Weights k/64 on integers < 2^8: one step is exact in FP64."""
    K = model.K_points(shape, d, r)
    rng = np.random.default_rng(34)
    wi = rng.integers(0, 9, size=K)
    w = wi / 64.0
    ui = rng.integers(0, 256, size=tuple(n + 2 * r for n in dims))
    got = oracle.step(shape, d, r, w, dims, ui.astype(float))
    offs = oracle.offsets(shape, d, r)
    inner = tuple(slice(r, r + n) for n in dims)
    acc = np.zeros(dims, dtype=np.int64)
    for k, o in enumerate(offs):
        acc += wi[k] * ui[tuple(slice(r + int(c), r + n + int(c)) for n, c in zip(dims, o))]
    assert np.array_equal(got[inner], acc / 64.0)


@pytest.mark.parametrize("shape,d,r,dims,steps", [("box", 2, 1, (16, 16), 8), ("star", 3, 2, (7, 6, 8), 5)])
def test_max_principle(shape, d, r, dims, steps):
    w, u = _problem(shape, d, r, dims, seed=35)
    assert np.all(w > 0) and abs(w.sum() - 1) < 1e-14
    got = oracle.run(shape, d, r, w, dims, u, steps)
    lo, hi = u.min(), u.max()
    tol = 1e-14
    assert got.min() >= lo - tol and got.max() <= hi + tol


# --- helpers used by the parity tests ------------------------------------------------

@pytest.mark.parametrize("shape,d,r,dims,steps,lo,hi", [
    ("box", 2, 3, (40, 37), 4, (0, 0), (5, 6)), ("box", 2, 3, (40, 37), 4, (17, 30), (23, 37)),
    ("star", 3, 2, (12, 11, 13), 3, (4, 0, 9), (8, 3, 13)), ("star", 2, 1, (9, 9), 0, (2, 2), (4, 5))])
def test_run_region_matches_full_run(shape, d, r, dims, steps, lo, hi):
    w, u = _problem(shape, d, r, dims, seed=36)
    full = oracle.run(shape, d, r, w, dims, u, steps)
    part = oracle.run_region(shape, d, r, w, dims, u, steps, lo, hi)
    box = tuple(slice(a + r, b + r) for a, b in zip(lo, hi))
    assert np.array_equal(part, full[box])


def test_thread_count_does_not_change_bits():
    w, u = _problem("box", 2, 2, (64, 45), seed=37)
    a = oracle.run("box", 2, 2, w, (64, 45), u, 6, nthreads=1)
    b = oracle.run("box", 2, 2, w, (64, 45), u, 6, nthreads=4)
    assert np.array_equal(a, b)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.run("box", 2, 1, np.ones(9) / 9, (4, 4), np.zeros((5, 6)), 1)
    with pytest.raises(ValueError):
        oracle.run("box", 2, 1, np.ones(9) / 9, (4, 4), np.zeros((6, 6)), -1)


def test_rel_linf():
    assert oracle.rel_linf(np.array([1.0, 2.0]), np.array([1.0, 2.0])) == 0.0
    assert oracle.rel_linf(np.array([1.0, 2.5]), np.array([1.0, 2.0])) == pytest.approx(0.25)
