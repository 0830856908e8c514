"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

This module holds no stencil arithmetic: it only draws weights and initial
fields.  Both the GPU path and the CPU oracle receive the very same arrays
from here, so neither side ever consumes numbers produced by the other.

Random numbers come from splitmix64, used as a counter-based generator: draw
i of seed s is mix(s + (i + 1) * 0x9E3779B97F4A7C15) with the published
splitmix64 finaliser, and a double in (0, 1) is ((x >> 11) + 0.5) * 2^-53.
Per problem the stream is used in this order: first the K weights (in the
lexicographic offset order the library uses), which are then divided by their
FP64 sum, then the interior field in row-major order.  The halo is 0.
"""
from __future__ import annotations

import concurrent.futures as cf
import math
import os

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the splitmix64 sequence of `seed`."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, count, _CHUNK):
            n = min(_CHUNK, count - c0)
            z = (np.arange(start + c0 + 1, start + c0 + 1 + n, dtype=np.uint64) * _GAMMA) + s
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            out[c0:c0 + n] = z ^ (z >> np.uint64(31))
    return out


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in (0, 1): ((x >> 11) + 0.5) * 2^-53.  Large draws are split
    over threads (each chunk is independent: the generator is counter-based)."""
    out = np.empty(count, dtype=np.float64)

    def fill(c0):
        n = min(_CHUNK, count - c0)
        x = splitmix64(seed, start + c0, n)
        out[c0:c0 + n] = ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)

    chunks = range(0, count, _CHUNK)
    if count > 4 * _CHUNK:
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(fill, chunks))
    else:
        for c0 in chunks:
            fill(c0)
    return out


def num_weights(shape: str, d: int, r: int) -> int:
    return (2 * r + 1) ** d if shape == "box" else 2 * d * r + 1


def weights(shape: str, d: int, r: int, seed: int) -> np.ndarray:
    """K weights drawn U(0,1) in offset order and divided by their FP64 sum."""
    w = uniform01(seed, 0, num_weights(shape, d, r))
    total = 0.0
    for x in w:  # fixed left-to-right order
        total += float(x)
    return w / total


def uniform_field(dims, r: int, seed: int, start: int, dtype=np.float64) -> np.ndarray:
    """Stored array (extents dims + 2r) with a zero halo and U(0,1) interior."""
    dims = tuple(int(n) for n in dims)
    stored = tuple(n + 2 * r for n in dims)
    u = np.zeros(stored, dtype=dtype)
    inner = tuple(slice(r, r + n) for n in dims)
    u[inner] = uniform01(seed, start, int(np.prod(dims))).reshape(dims).astype(dtype)
    return u


def sine_field(dims, r: int, seed: int, start: int, dtype=np.float32, modes: int = 8) -> np.ndarray:
    """Smooth 2-D field: sum of `modes` seeded sine modes plus 1e-3 uniform noise.

    Per mode m: amplitude a_m = U/8, integer wavenumbers k_y, k_x in 1..16 and a
    phase U * 2 pi; f = sum_m a_m sin(2 pi (k_y y / N_y + k_x x / N_x) + phi_m)
    + 1e-3 U, computed in FP64 and rounded to the storage type.
    """
    ny, nx = (int(n) for n in dims)
    p = uniform01(seed, start, 4 * modes)
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    f = np.zeros((ny, nx), dtype=np.float64)
    for m in range(modes):
        a = p[4 * m] / 8.0
        ky = 1 + int(p[4 * m + 1] * 16.0)
        kx = 1 + int(p[4 * m + 2] * 16.0)
        phi = p[4 * m + 3] * 2.0 * math.pi
        f += a * np.sin(2.0 * math.pi * (ky * y / ny + kx * x / nx) + phi)
    f += 1e-3 * uniform01(seed, start + 4 * modes, ny * nx).reshape(ny, nx)
    u = np.zeros((ny + 2 * r, nx + 2 * r), dtype=dtype)
    u[r:r + ny, r:r + nx] = f.astype(dtype)
    return u


def problem(shape: str, d: int, r: int, dims, seed: int, dtype=np.float64, field: str = "uniform"):
    """(weights FP64, stored initial field in `dtype`) for one seeded problem."""
    w = weights(shape, d, r, seed)
    K = len(w)
    if field == "uniform":
        u = uniform_field(dims, r, seed, K, dtype)
    elif field == "sine":
        u = sine_field(dims, r, seed, K, dtype)
    else:
        raise ValueError(field)
    return w, u


BATCH_KINDS = (("star", 1), ("star", 2), ("box", 1), ("box", 3))


def batch_descs(n: int = 512, seed: int = 5, lo: int = 64, hi: int = 4096):
    """Uneven 2-D batch: per grid two sides round(exp(U(ln lo, ln hi))) and a
    stencil drawn uniformly from BATCH_KINDS.  Draw order per grid: ny, nx, kind.
    Returns a list of (shape, r, ny, nx, field_seed)."""
    p = uniform01(seed, 0, 3 * n)
    out = []
    for g in range(n):
        ny = int(round(math.exp(math.log(lo) + p[3 * g] * (math.log(hi) - math.log(lo)))))
        nx = int(round(math.exp(math.log(lo) + p[3 * g + 1] * (math.log(hi) - math.log(lo)))))
        shape, r = BATCH_KINDS[min(int(p[3 * g + 2] * len(BATCH_KINDS)), len(BATCH_KINDS) - 1)]
        out.append((shape, r, ny, nx, seed * 1000003 + g))
    return out
