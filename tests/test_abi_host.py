"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/gbstencil.h declares, validates arguments, and its
model (the dispatch rule) agrees with the oracle's copy of the paper's model.
No test here launches a kernel."""
import ctypes
import itertools

import pytest

from oracle import model
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import build as gbuild


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return B.load()


def test_exports_every_declared_symbol(lib):
    names = B.declared_symbols()
    assert "stencil_plan_create" in names and "stencil_run" in names and "stencil_plan_destroy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    for s in range(7):
        assert B.stencil_status_string(s) != "unknown status"
    assert B.stencil_status_string(0) == "ok"
    assert B.stencil_status_string(7) == "unknown status"


@pytest.mark.parametrize("kind,status", [("bad_alloc", B.STENCIL_ERR_OOM),
                                         ("runtime", B.STENCIL_ERR_INTERNAL)])
def test_exception_stops_at_the_boundary(lib, kind, status):
    """A C++ exception thrown inside the library (planted by a test hook)
    comes back as a status and a message, the process keeps running and the
    plan stays usable and unchanged."""
    p = B.stencil_plan_create("box", 2, 1, _w("box", 2, 1), "f64", (64, 64), 2)
    try:
        before = B.stencil_plan_info(p)
        rc = lib.stencil_plan_set_option(p, b"debug_host_exception", kind.encode())
        assert rc == status
        msg = B.stencil_last_error()
        assert msg.startswith("stencil_plan_set_option: ")
        if kind == "runtime":
            assert "planted by debug_host_exception" in msg
        assert B.stencil_plan_info(p) == before
        B.stencil_plan_set_option(p, "t", 1)
        assert B.stencil_plan_info(p)["t"] == 1
    finally:
        B.stencil_plan_destroy(p)


def _w(shape, d, r):
    return [1.0 / model.K_points(shape, d, r)] * model.K_points(shape, d, r)


@pytest.mark.parametrize("args,status", [
    (("box", 1, 1, "f64", (8,)), B.STENCIL_ERR_INVALID_ARG),        # d = 1
    (("box", 4, 1, "f64", (8, 8, 8, 8)), B.STENCIL_ERR_INVALID_ARG),  # d = 4
    (("box", 2, 0, "f64", (8, 8)), B.STENCIL_ERR_INVALID_ARG),      # r = 0
    (("box", 2, 1, "f64", (0, 8)), B.STENCIL_ERR_INVALID_ARG),      # empty extent
    (("box", 2, 1, "f64", (-3, 8)), B.STENCIL_ERR_INVALID_ARG),
    (("box", 3, 3, "f64", (8, 8, 8)), B.STENCIL_ERR_UNSUPPORTED),   # no 3-D box r=3 kernel
    (("box", 2, 9, "f32", (64, 64)), B.STENCIL_ERR_UNSUPPORTED),
])
def test_plan_create_rejects(lib, args, status):
    shape, d, r, dt, dims = args
    K = model.K_points(shape, max(d, 1), max(r, 1)) if 1 <= d <= 3 else 1
    with pytest.raises(B.StencilError) as e:
        B.stencil_plan_create(shape, d, r, [0.1] * K, dt, dims, 0)
    assert e.value.status == status


def test_plan_create_rejects_nonfinite_and_bad_t(lib):
    w = _w("box", 2, 1)
    w[3] = float("nan")
    with pytest.raises(B.StencilError):
        B.stencil_plan_create("box", 2, 1, w, "f64", (8, 8), 0)
    with pytest.raises(B.StencilError):
        B.stencil_plan_create("box", 2, 1, _w("box", 2, 1), "f64", (8, 8), 17)


def test_null_pointer_arguments(lib):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(8, 8)
    assert lib.stencil_plan_create(None, 0, 2, 1, (ctypes.c_double * 9)(), 0, dims, 0) == B.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_plan_create(ctypes.byref(h), 0, 2, 1, None, 0, dims, 0) == B.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_run(None, None, None, 1, None) == B.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_plan_info(None, None) == B.STENCIL_ERR_INVALID_ARG
    lib.stencil_plan_destroy(None)


def test_run_argument_checks_launch_nothing(lib):
    p = B.stencil_plan_create("box", 2, 1, _w("box", 2, 1), "f64", (8, 8), 1)
    try:
        n0 = B.stencil_launch_count()
        with pytest.raises(B.StencilError) as e:
            B.stencil_run(p, 4096, 4096, 3, 0)  # in == out
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:
            B.stencil_run(p, 4096, 1 << 20, -1, 0)
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:  # overlapping buffers
            B.stencil_run(p, 4096, 4096 + 8, 3, 0)
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:  # > 1 sweep without workspace
            B.stencil_run(p, 4096, 1 << 20, 3, 0)
        assert e.value.status == B.STENCIL_ERR_OOM
        with pytest.raises(B.StencilError) as e:
            B.stencil_run_host(p, 4096, 1 << 20, 1, 0)
        assert e.value.status == B.STENCIL_ERR_OOM
        for steps, reps in ((0, 1), (3, 0)):  # the autotuner checks before any CUDA call
            with pytest.raises(B.StencilError) as e:
                B.stencil_plan_autotune(p, 4096, 1 << 20, steps, reps, 0)
            assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        assert lib.stencil_plan_autotune(None, None, None, 1, 1, None, None, 0, None) == B.STENCIL_ERR_INVALID_ARG
        assert B.stencil_launch_count() == n0
    finally:
        B.stencil_plan_destroy(p)


def test_workspace_bytes(lib):
    p = B.stencil_plan_create("star", 3, 2, _w("star", 3, 2), "f32", (5, 6, 7), 1)
    try:
        g = 9 * 10 * 11 * 4
        assert B.stencil_plan_workspace_bytes(p) == g
        assert B.stencil_plan_workspace_bytes(p, True) == 3 * g
    finally:
        B.stencil_plan_destroy(p)


def test_options(lib):
    p = B.stencil_plan_create("box", 2, 2, _w("box", 2, 2), "f32", (100, 200), 0)
    try:
        B.stencil_plan_set_option(p, "t", "3")
        assert B.stencil_plan_info(p)["t"] == 3
        B.stencil_plan_set_option(p, "tile", "32x64")
        assert B.stencil_plan_info(p)["tile"] == [1, 32, 64]
        B.stencil_plan_set_option(p, "path", "cuda_core")
        for k, v in (("nope", "1"), ("t", "99"), ("path", "fpga"), ("tile", "3x5x7"), ("precision", "fp8")):
            with pytest.raises(B.StencilError) as e:
                B.stencil_plan_set_option(p, k, v)
            assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        assert B.stencil_plan_info(p)["t"] == 3  # failed options leave the plan unchanged
    finally:
        B.stencil_plan_destroy(p)


def test_fp64_rejects_reduced_precision(lib):
    p = B.stencil_plan_create("box", 2, 3, _w("box", 2, 3), "f64", (64, 64), 0)
    try:
        with pytest.raises(B.StencilError):
            B.stencil_plan_set_option(p, "precision", "tf32")
    finally:
        B.stencil_plan_destroy(p)


# ---- the product's model against the oracle's ---------------------------------------

@pytest.mark.parametrize("shape,d,r,t,D,S,beta", list(itertools.product(
    ("box", "star"), (2, 3), (1, 2, 3), (1, 2, 4, 7), (4, 8), (0.3125, 0.5, 1.0), (1.0, 3.0)))[::7])
def test_model_matches_oracle_model(lib, shape, d, r, t, D, S, beta):
    P_cu, P_tc, Bw = 80e12, 1.1e15, 6.8e12
    got = B.stencil_model_predict(shape, d, r, t, D, S, beta, P_cu, P_tc, Bw)
    assert got["K"] == model.K_points(shape, d, r)
    assert got["K_fused"] == model.K_fused(shape, d, r, t)
    assert got["alpha"] == pytest.approx(model.alpha(shape, d, r, t), rel=1e-14)
    assert got["I_cu"] == pytest.approx(model.I_cu(shape, d, r, t, D), rel=1e-14)
    assert got["I_tc"] == pytest.approx(model.I_tc(shape, d, r, t, D, S, beta), rel=1e-14)
    assert got["C_tc"] == pytest.approx(model.C_tc(shape, d, r, t, S, beta), rel=1e-14)
    assert got["P_tc_actual"] == pytest.approx(model.P_tc_actual(shape, d, r, t, D, S, P_tc, Bw, beta), rel=1e-14)
    assert got["P_cu_actual"] == pytest.approx(model.P_cu_actual(shape, d, r, t, D, P_cu, Bw), rel=1e-14)
    assert got["scenario"] == model.scenario(shape, d, r, t, D, S, P_cu, P_tc, Bw, beta)
    assert bool(got["sweet_spot"]) == model.in_sweet_spot(shape, d, r, t, D, S, P_cu, P_tc, Bw, beta)
    assert got["gstencils_cu"] * 1e9 == pytest.approx(model.gstencils_roof_cu(shape, d, r, t, D, P_cu, Bw))


def test_model_rejects_bad_input(lib):
    for bad in (dict(sparsity=0.0), dict(sparsity=1.5), dict(t=0), dict(B=0.0), dict(beta=0.5)):
        args = dict(shape="box", d=2, r=1, t=1, dtype_bytes=8, sparsity=0.5, beta=1.0, P_cu=1e12, P_tc=2e12, B=1e12)
        args.update(bad)
        with pytest.raises(B.StencilError):
            B.stencil_model_predict(**args)


def test_peaks_roundtrip(lib):
    old = B.stencil_get_peaks()
    try:
        B.stencil_set_peaks(hbm_bytes_per_s=1.0e12)
        assert B.stencil_get_peaks()["hbm_bytes_per_s"] == 1.0e12
        assert B.stencil_get_peaks()["cu_f64_flops"] == old["cu_f64_flops"]  # zero fields unchanged
        B.stencil_set_peaks(sptc_bf16_flops=7.0e15)  # the last field of the table
        assert B.stencil_get_peaks()["sptc_bf16_flops"] == 7.0e15
        for bad in (-1.0, float("nan"), float("inf")):
            before = B.stencil_get_peaks()
            with pytest.raises(B.StencilError):
                B.stencil_set_peaks(cu_f32_flops=1e14, tc_tf32_flops=bad)
            assert B.stencil_get_peaks() == before  # refused as a whole
    finally:
        B.stencil_set_peaks(**old)


def test_peaks_table_is_thread_safe(lib):
    """Threads replacing the table while others create plans and read it
    never see a torn table: every read is one of the tables written."""
    import threading
    old = B.stencil_get_peaks()
    tables = [dict(old, hbm_bytes_per_s=h, cu_f64_flops=h / 5) for h in (2e12, 4e12, 8e12)]
    seen, stop = [], threading.Event()

    def writer():
        i = 0
        while not stop.is_set():
            B.stencil_set_peaks(**tables[i % 3])
            i += 1

    def reader():
        for _ in range(300):
            p = B.stencil_get_peaks()
            seen.append(p["cu_f64_flops"] * 5 == p["hbm_bytes_per_s"])
            h = B.stencil_plan_create("box", 2, 1, _w("box", 2, 1), "f64", (64, 64), 0)
            B.stencil_plan_destroy(h)

    try:
        ws = [threading.Thread(target=writer) for _ in range(2)]
        rs = [threading.Thread(target=reader) for _ in range(2)]
        for th in ws + rs:
            th.start()
        for th in rs:
            th.join()
        stop.set()
        for th in ws:
            th.join()
        assert seen and all(seen)
    finally:
        B.stencil_set_peaks(**old)


def test_dispatch_fp64_picks_cuda_cores_t1(lib):
    """With GB300's FP64 rate every FP64 configuration is compute-bound at
    t=1 (ridge ~0.19 FLOP/B), so fusion cannot help and the CUDA-core t=1
    plan is the fastest (ties go to CUDA cores and smaller t)."""
    p = B.stencil_plan_create("box", 2, 3, _w("box", 2, 3), "f64", (16384, 16384), 0)
    try:
        info = B.stencil_plan_info(p)
        assert info["path"] == B.PATH_CUDA_CORE and info["t"] == 1
        assert info["memory_bound"] == 0
        assert info["intensity"] == pytest.approx(49 / 8)
    finally:
        B.stencil_plan_destroy(p)


def test_dispatch_fp32_paper_model_and_issue_roof(lib):
    """Box-2D2R FP32 on CUDA cores.  The paper's model (Eq. 8, no instruction
    costs) classifies it memory-bound at t = 1 (I = 6.25 against a ridge of
    80.5 TFLOP/s / 6.8 TB/s = 11.8) and compute-bound from t = 2.  The
    FP32 sub-step this library runs is issue-bound instead (25 FMAs and ~19
    other instructions per output at 53.5 % issue): its issue roof,
    t * 152 * 2.07e9 / (overlap * t * (25 + 19) / (128 * 0.535)), is below
    58 % of the HBM roof 6.8e12 / 8 = 850 G (where the one-step sweep
    saturates) and falls with t through the overlap, so the dispatcher keeps
    t = 1 (measured on GB300: 490 at t = 1, 488 at t = 2 GStencil/s)."""
    pk = B.stencil_get_peaks()
    m1 = B.stencil_model_predict("box", 2, 2, 1, 4, 1.0, 1.0, pk["cu_f32_flops"], pk["cu_f32_flops"],
                                 pk["hbm_bytes_per_s"])
    m2 = B.stencil_model_predict("box", 2, 2, 2, 4, 1.0, 1.0, pk["cu_f32_flops"], pk["cu_f32_flops"],
                                 pk["hbm_bytes_per_s"])
    assert m1["I_cu"] < m1["ridge_cu"] <= m2["I_cu"]
    p = B.stencil_plan_create("box", 2, 2, _w("box", 2, 2), "f32", (16384, 16384), 0)
    try:
        info = B.stencil_plan_info(p)
        assert info["path"] == B.PATH_CUDA_CORE and info["t"] == 1
        issue_roof = 152 * 2.07e9 / ((25 + 19) / (128 * 0.535)) / 1e9
        assert issue_roof < 0.58 * pk["hbm_bytes_per_s"] / 8 / 1e9
        assert info["predicted_gstencils"] == pytest.approx(issue_roof, rel=1e-6)
        assert info["predicted_gstencils"] < pk["hbm_bytes_per_s"] / 8 / 1e9
    finally:
        B.stencil_plan_destroy(p)


# ---- batched form (host side) ---------------------------------------------------------

def test_batch_create_validation(lib):
    w9 = _w("box", 2, 1)
    with pytest.raises(B.StencilError) as e:
        B.stencil_batch_create([], "f32")
    assert e.value.status == B.STENCIL_ERR_INVALID_ARG
    with pytest.raises(B.StencilError) as e:
        B.stencil_batch_create([("box", 4, 10, 10, _w("box", 2, 4))], "f32")
    assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
    with pytest.raises(B.StencilError) as e:
        B.stencil_batch_create([("box", 1, 0, 10, w9)], "f32")
    assert e.value.status == B.STENCIL_ERR_INVALID_ARG


def test_batch_workspace_and_no_launch_without_it(lib):
    grids = [("box", 1, 100, 120, _w("box", 2, 1)), ("star", 2, 33, 7, _w("star", 2, 2))]
    h = B.stencil_batch_create(grids, "f32", 2)
    try:
        one = B.stencil_batch_workspace_bytes(h, 2)   # one sweep each: no ping-pong grids
        many = B.stencil_batch_workspace_bytes(h, 9)
        assert many > one > 0
        assert many - one >= (102 * 122 + 37 * 11) * 4  # a ping-pong grid per grid
        assert B.stencil_batch_info(h, 0)["t"] == 2
        n0 = B.stencil_launch_count()
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_run(h, [4096, 8192], [1 << 20, 1 << 21], 9, 0)
        assert e.value.status == B.STENCIL_ERR_OOM
        # the autotuner refuses the same way, and bad counts, before any CUDA call
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_autotune(h, [4096, 8192], [1 << 20, 1 << 21], 9, 1, 0)
        assert e.value.status == B.STENCIL_ERR_OOM
        for steps, reps in ((0, 1), (9, 0)):
            with pytest.raises(B.StencilError) as e:
                B.stencil_batch_autotune(h, [4096, 8192], [1 << 20, 1 << 21], steps, reps, 0)
            assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:  # a grid's in and out are the same buffer
            B.stencil_batch_run(h, [4096, 8192], [4096, 1 << 21], 9, 0)
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        assert B.stencil_launch_count() == n0
    finally:
        B.stencil_batch_destroy(h)


def test_batch_precision_and_path_options(lib):
    grids = [("box", 2, 300, 310, _w("box", 2, 2)), ("star", 1, 40, 70, _w("star", 2, 1))]
    h = B.stencil_batch_create(grids, "f32", 0)
    try:
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_set_option(h, "precision", "fp8")
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:  # FP32 native has no tensor-core form
            B.stencil_batch_set_option(h, "path", "tensor_core")
        assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
        assert B.stencil_batch_info(h, 0)["path"] == B.PATH_CUDA_CORE  # unchanged after the refusal
        B.stencil_batch_set_option(h, "precision", "tf32x3")
        B.stencil_batch_set_option(h, "path", "tensor_core")
        for i in range(2):
            info = B.stencil_batch_info(h, i)
            assert info["path"] == B.PATH_TENSOR_CORE and info["precision"] == B.PREC_TF32X3
        B.stencil_batch_set_option(h, "path", "cuda_core")
        assert B.stencil_batch_info(h, 1)["path"] == B.PATH_CUDA_CORE
        n0 = B.stencil_launch_count()
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_autotune(h, [4096, 8192], [1 << 20, 1 << 21], 0, stream=0)
        assert e.value.status == B.STENCIL_ERR_INVALID_ARG
        with pytest.raises(B.StencilError) as e:  # no workspace
            B.stencil_batch_autotune(h, [4096, 8192], [1 << 20, 1 << 21], 5, stream=0)
        assert e.value.status == B.STENCIL_ERR_OOM
        assert B.stencil_launch_count() == n0
    finally:
        B.stencil_batch_destroy(h)
    h64 = B.stencil_batch_create(grids, "f64", 0)
    try:
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_set_option(h64, "precision", "tf32")
        assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
        B.stencil_batch_set_option(h64, "path", "tensor_core")  # FP64 MMA
        assert B.stencil_batch_info(h64, 0)["path"] == B.PATH_TENSOR_CORE
    finally:
        B.stencil_batch_destroy(h64)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,r", [("star", 2), ("box", 1)])
def test_dispatch_3d_keeps_one_step_per_sweep(lib, dtype, shape, r):
    """3-D: the dispatcher's own choice is t = 1 (the streaming kernel; fused
    3-D tiles re-read their halo volume); an explicit t is still honoured."""
    w = _w(shape, 3, r)
    h = B.stencil_plan_create(shape, 3, r, w, dtype, (512, 512, 512), 0)
    try:
        info = B.stencil_plan_info(h)
        assert info["path"] == B.PATH_CUDA_CORE and info["t"] == 1
        assert list(info["tile"]) == [64, 16 if dtype == "f64" else 32, 64]
    finally:
        B.stencil_plan_destroy(h)
    h = B.stencil_plan_create(shape, 3, r, w, dtype, (512, 512, 512), 2)
    try:
        assert B.stencil_plan_info(h)["t"] == 2
    finally:
        B.stencil_plan_destroy(h)


def test_batch_refuses_more_work_items_than_an_int_indexes(lib):
    """2^31 steps of a one-tile grid at t = 1 is more (grid, tile, sweep) items
    than the device tables index: refused before any upload or launch."""
    h = B.stencil_batch_create([("star", 1, 16, 16, _w("star", 2, 1))], "f32", 1)
    try:
        n0 = B.stencil_launch_count()
        with pytest.raises(B.StencilError) as e:
            B.stencil_batch_run(h, [4096], [1 << 20], 1 << 31, 0)
        assert e.value.status == B.STENCIL_ERR_UNSUPPORTED
        assert B.stencil_launch_count() == n0
    finally:
        B.stencil_batch_destroy(h)


def test_host_alloc_argument_checks_without_cuda(lib):
    """stencil_host_alloc / stencil_host_free refuse bad arguments before any
    CUDA call (the allocation itself needs a GPU: tests/test_gpu_host_buffer.py)."""
    import ctypes
    L = B.load()
    p = ctypes.c_void_p()
    assert L.stencil_host_alloc(None, 4096) == B.STENCIL_ERR_INVALID_ARG
    assert L.stencil_host_alloc(ctypes.byref(p), 0) == B.STENCIL_ERR_INVALID_ARG
    assert L.stencil_host_free(None) == B.STENCIL_OK
    buf = ctypes.create_string_buffer(64)
    assert L.stencil_host_free(ctypes.addressof(buf)) == B.STENCIL_ERR_INVALID_ARG
