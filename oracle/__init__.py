"""Plain FP64 CPU oracle for repeated star/box stencil sweeps.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import
this package.  The GPU product path (package ``paper_2603_00477_gb300``) never
imports it, and the two share no code: the arithmetic lives in ``oracle.c``
(stencil sweeps, composite kernel) and ``model.py`` (the paper's performance
model), both written from the paper.

Functions here take and return numpy arrays; the arithmetic is in C (FP64,
``-ffp-contract=off``, fixed summation order), built with gcc by
:func:`build`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

BOX, STAR = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_num_offsets.argtypes = [ctypes.c_int] * 3
        lib.oracle_offsets.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
        lib.oracle_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64p, dp, dp, ctypes.c_int]
        lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64p, dp, ctypes.c_int64,
                                   ctypes.c_int]
        lib.oracle_compose.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.oracle_apply_dense.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, i64p, dp, dp,
                                           ctypes.c_int, ctypes.c_int]
        lib.oracle_run_region.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, i64p, dp, ctypes.c_int64,
                                          i64p, i64p, dp, ctypes.c_int]
        lib.oracle_max_threads.argtypes = []
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64(seq) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(seq, dtype=np.int64))


def _check(rc: int, what: str):
    if rc < 0:
        raise ValueError(f"oracle: {what} rejected its arguments (rc={rc})")


def shape_code(shape) -> int:
    if isinstance(shape, str):
        return {"box": BOX, "star": STAR}[shape.lower()]
    return int(shape)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def num_offsets(shape, d: int, r: int) -> int:
    k = _load().oracle_num_offsets(shape_code(shape), d, r)
    _check(k, "num_offsets")
    return k


def offsets(shape, d: int, r: int) -> np.ndarray:
    """The K offsets in O order (lexicographic, first axis outermost)."""
    K = num_offsets(shape, d, r)
    out = np.zeros((K, d), dtype=np.int32)
    _load().oracle_offsets(shape_code(shape), d, r, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def _field(u: np.ndarray, dims, r: int) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    want = tuple(int(n) + 2 * r for n in dims)
    if u.shape != want:
        raise ValueError(f"oracle: field shape {u.shape} != stored extents {want}")
    return u


def step(shape, d, r, w, dims, u, nthreads: int = 0) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = _field(u, dims, r)
    v = np.empty_like(u)
    _check(_load().oracle_step(shape_code(shape), d, r, _dp(w), _i64(dims).ctypes.data_as(
        ctypes.POINTER(ctypes.c_int64)), _dp(u), _dp(v), nthreads), "step")
    return v


def run(shape, d, r, w, dims, u, steps: int, nthreads: int = 0) -> np.ndarray:
    """`steps` stepwise sweeps; returns a new FP64 stored array (halo kept)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = _field(u, dims, r).copy()
    dims64 = _i64(dims)
    _check(_load().oracle_run(shape_code(shape), d, r, _dp(w), dims64.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int64)), _dp(out), int(steps), nthreads), "run")
    return out


def compose(shape, d, r, w, t: int) -> np.ndarray:
    """Dense composite kernel w^(t), shape (2tr+1,)*d."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    side = 2 * t * r + 1
    wt = np.zeros((side,) * d, dtype=np.float64)
    _check(_load().oracle_compose(shape_code(shape), d, r, _dp(w), int(t), _dp(wt)), "compose")
    return wt


def apply_dense(d, wk, halo, dims, u, margin, nthreads: int = 0, v=None) -> np.ndarray:
    """One sweep of a dense kernel wk (radius R) at points >= margin from the boundary."""
    wk = np.ascontiguousarray(wk, dtype=np.float64)
    R = (wk.shape[0] - 1) // 2
    u = _field(u, dims, halo)
    v = u.copy() if v is None else np.ascontiguousarray(v, dtype=np.float64)
    _check(_load().oracle_apply_dense(d, R, _dp(wk), halo, _i64(dims).ctypes.data_as(
        ctypes.POINTER(ctypes.c_int64)), _dp(u), _dp(v), int(margin), nthreads), "apply_dense")
    return v


def run_region(shape, d, r, w, dims, u, steps: int, lo, hi, nthreads: int = 0) -> np.ndarray:
    """`steps` stepwise sweeps evaluated only on the dependency cone of the
    interior box [lo, hi); returns that box."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = _field(u, dims, r)
    lo64, hi64 = _i64(lo), _i64(hi)
    out = np.zeros(tuple(int(b - a) for a, b in zip(lo64, hi64)), dtype=np.float64)
    _check(_load().oracle_run_region(
        shape_code(shape), d, r, _dp(w), _i64(dims).ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(u),
        int(steps), lo64.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
        hi64.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out), nthreads), "run_region")
    return out


def rel_linf(got: np.ndarray, ref: np.ndarray) -> float:
    """Normwise relative L-infinity error max|g - o| / max|o| (0 when both vanish)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    if den == 0.0:
        return num
    return num / den
