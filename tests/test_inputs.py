"""Pins of the seeded input generator that both the oracle and the GPU path
read from: splitmix64 as published (a scalar implementation with Python
integers, and the first output of state 0), its counter-based property across
the chunk boundary of the vectorised form, the (0, 1) double mapping, and the
problem layout (normalised weights first, zero halo)."""
import numpy as np

from paper_2603_00477_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix64_scalar(seed, n):
    """The published generator: x += 0x9E3779B97F4A7C15, then the finaliser."""
    x, out = seed & MASK, []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & MASK
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_first_output_of_state_zero():
    assert int(inputs.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF


def test_matches_scalar_definition():
    for seed in (0, 1, 5, 123456789, (1 << 64) - 1):
        want = splitmix64_scalar(seed, 300)
        got = [int(v) for v in inputs.splitmix64(seed, 0, 300)]
        assert got == want, seed


def test_counter_based_across_chunks():
    n = (1 << 22) + 5  # crosses the vectorised chunk size
    full = inputs.splitmix64(7, 0, n)
    tail = inputs.splitmix64(7, (1 << 22) - 3, 8)
    assert np.array_equal(full[(1 << 22) - 3:(1 << 22) + 5], tail)
    assert [int(v) for v in full[-3:]] == splitmix64_scalar(7, n)[-3:]


def test_uniform_mapping():
    x = inputs.splitmix64(3, 10, 1000)
    u = inputs.uniform01(3, 10, 1000)
    assert np.array_equal(u, ((x >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53)
    assert u.min() > 0.0 and u.max() < 1.0


def test_problem_layout():
    w, u = inputs.problem("box", 2, 2, (7, 9), seed=4, dtype=np.float64)
    assert w.shape == (25,) and abs(w.sum() - 1.0) < 1e-15 and (w > 0).all()
    raw = inputs.uniform01(4, 0, 25)  # the K weights are the first draws
    total = 0.0
    for x in raw:  # summed left to right, as documented
        total += float(x)
    assert np.array_equal(w, raw / total)
    assert u.shape == (11, 13)
    # the interior follows the weights in the stream, row-major
    assert np.array_equal(u[2:9, 2:11], inputs.uniform01(4, 25, 63).reshape(7, 9))
    halo = np.ones(u.shape, bool)
    halo[2:9, 2:11] = False
    assert not u[halo].any()
    assert (u[~halo] > 0).all() and (u[~halo] < 1).all()
