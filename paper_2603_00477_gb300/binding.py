"""Thin Python binding of libgbstencil's C ABI (include/gbstencil.h).

Argument marshalling only: every step of the stencil runs in the library's
CUDA kernels.  Functions carry the C names.  Device buffers are PyTorch CUDA
tensors (their data pointers are passed through), streams are torch streams
(or raw cudaStream_t integers).  There is no CPU fallback: if the compiled
library is missing, loading fails with an error naming the build step.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

_LIB = None

STENCIL_OK, STENCIL_ERR_INVALID_ARG, STENCIL_ERR_UNSUPPORTED, STENCIL_ERR_CUDA, STENCIL_ERR_OOM, \
    STENCIL_ERR_TIMEOUT, STENCIL_ERR_INTERNAL = range(7)
BOX, STAR = 0, 1
F64, F32 = 0, 1
PATH_AUTO, PATH_CUDA_CORE, PATH_TENSOR_CORE, PATH_SPARSE_TENSOR_CORE = range(4)
PREC_NATIVE, PREC_TF32, PREC_TF32X3, PREC_BF16X3, PREC_ANY, PREC_OZAKI, PREC_F16, PREC_F16X3 = range(8)
PATH_NAMES = {0: "auto", 1: "cuda_core", 2: "tensor_core", 3: "sparse_tensor_core"}
PREC_NAMES = {0: "native", 1: "tf32", 2: "tf32x3", 3: "bf16x3", 4: "any", 5: "ozaki", 6: "f16", 7: "f16x3"}


class StencilError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[{status}] {msg}")
        self.status = status


class stencil_peaks(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "hbm_bytes_per_s", "cu_f64_flops", "cu_f32_flops", "tc_f64_flops", "tc_tf32_flops", "tc_bf16_flops",
        "sptc_tf32_flops", "sptc_bf16_flops")]


class stencil_info(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("precision", ctypes.c_int), ("t", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("K", ctypes.c_int), ("K_fused", ctypes.c_int),
                ("alpha", ctypes.c_double), ("sparsity", ctypes.c_double), ("beta", ctypes.c_double),
                ("intensity", ctypes.c_double), ("ridge", ctypes.c_double), ("scenario", ctypes.c_int),
                ("memory_bound", ctypes.c_int), ("predicted_gstencils", ctypes.c_double),
                ("predicted_cu_gstencils", ctypes.c_double), ("predicted_tc_gstencils", ctypes.c_double)]


class stencil_tc_layout(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int), ("n_tile", ctypes.c_int), ("k_inst", ctypes.c_int), ("kext", ctypes.c_int),
                ("nkb", ctypes.c_int), ("sparsity", ctypes.c_double)]


class stencil_grid_desc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("r", ctypes.c_int), ("ny", ctypes.c_int64), ("nx", ctypes.c_int64),
                ("weights", ctypes.POINTER(ctypes.c_double))]


class stencil_sptc_layout(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int), ("nc", ctypes.c_int), ("ns", ctypes.c_int), ("sigma", ctypes.c_int),
                ("sparsity", ctypes.c_double)]


class stencil_batch_tune_result(ctypes.Structure):
    _fields_ = [("cls", ctypes.c_int), ("shape", ctypes.c_int), ("r", ctypes.c_int), ("size_class", ctypes.c_int),
                ("ngrids", ctypes.c_int), ("path", ctypes.c_int), ("precision", ctypes.c_int), ("t", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("tile_x", ctypes.c_int), ("model_gstencils", ctypes.c_double),
                ("measured_gstencils", ctypes.c_double), ("chosen", ctypes.c_int)]


class stencil_tune_result(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("precision", ctypes.c_int), ("t", ctypes.c_int),
                ("model_gstencils", ctypes.c_double), ("measured_gstencils", ctypes.c_double),
                ("tile_y", ctypes.c_int), ("tile_x", ctypes.c_int)]


class stencil_model_in(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int), ("d", ctypes.c_int), ("r", ctypes.c_int), ("t", ctypes.c_int),
                ("dtype_bytes", ctypes.c_int), ("sparsity", ctypes.c_double), ("beta", ctypes.c_double),
                ("P_cu", ctypes.c_double), ("P_tc", ctypes.c_double), ("B", ctypes.c_double)]


class stencil_model_out(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("K_fused", ctypes.c_int), ("alpha", ctypes.c_double),
                ("C_cu", ctypes.c_double), ("C_tc", ctypes.c_double), ("M", ctypes.c_double),
                ("I_cu", ctypes.c_double), ("I_tc", ctypes.c_double), ("ridge_cu", ctypes.c_double),
                ("ridge_tc", ctypes.c_double), ("P_cu_actual", ctypes.c_double), ("P_tc_actual", ctypes.c_double),
                ("speedup", ctypes.c_double), ("scenario", ctypes.c_int), ("sweet_spot", ctypes.c_int),
                ("gstencils_cu", ctypes.c_double), ("gstencils_tc", ctypes.c_double)]


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load the in-tree libgbstencil.so (built by __graft_entry__.build())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libgbstencil.so is not built ({path}); run `python -c 'import __graft_entry__ as g; "
                          f"g.build()'` (needs nvcc, CUDA 13, sm_103a)")
    L = ctypes.CDLL(path)
    vp, i64, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.stencil_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(i64), ctypes.c_int]
    L.stencil_plan_create.restype = st
    L.stencil_plan_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    L.stencil_plan_set_option.restype = st
    L.stencil_plan_info.argtypes = [vp, ctypes.POINTER(stencil_info)]
    L.stencil_plan_info.restype = st
    L.stencil_plan_workspace_bytes.argtypes = [vp, ctypes.c_int]
    L.stencil_plan_workspace_bytes.restype = ctypes.c_size_t
    L.stencil_plan_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.stencil_plan_set_workspace.restype = st
    L.stencil_run.argtypes = [vp, vp, vp, i64, vp]
    L.stencil_run.restype = st
    L.stencil_run_noalloc.argtypes = [vp, vp, vp, i64, vp]
    L.stencil_run_noalloc.restype = st
    L.stencil_run_host.argtypes = [vp, vp, vp, i64, vp]
    L.stencil_run_host.restype = st
    L.stencil_host_alloc.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t]
    L.stencil_host_alloc.restype = st
    L.stencil_host_free.argtypes = [vp]
    L.stencil_host_free.restype = st
    L.stencil_plan_sptc_layout.argtypes = [vp, ctypes.c_int, ctypes.POINTER(stencil_sptc_layout), vp, vp, vp, vp, vp]
    L.stencil_plan_sptc_layout.restype = st
    L.stencil_plan_autotune.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.POINTER(stencil_tune_result),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.stencil_plan_autotune.restype = st
    L.stencil_plan_destroy.argtypes = [vp]
    L.stencil_plan_destroy.restype = None
    L.stencil_model_predict.argtypes = [ctypes.POINTER(stencil_model_in), ctypes.POINTER(stencil_model_out)]
    L.stencil_model_predict.restype = st
    L.stencil_set_peaks.argtypes = [ctypes.POINTER(stencil_peaks)]
    L.stencil_set_peaks.restype = st
    L.stencil_get_peaks.argtypes = [ctypes.POINTER(stencil_peaks)]
    L.stencil_get_peaks.restype = st
    L.stencil_probe_peaks.argtypes = [ctypes.POINTER(stencil_peaks), vp]
    L.stencil_probe_peaks.restype = st
    L.stencil_plan_tc_layout.argtypes = [vp, ctypes.c_int, ctypes.POINTER(stencil_tc_layout),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]
    L.stencil_plan_tc_layout.restype = st
    L.stencil_device_status.argtypes = [vp]
    L.stencil_device_status.restype = st
    L.stencil_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(stencil_grid_desc),
                                       ctypes.c_int, ctypes.c_int]
    L.stencil_batch_create.restype = st
    L.stencil_batch_workspace_bytes.argtypes = [vp, i64]
    L.stencil_batch_workspace_bytes.restype = ctypes.c_size_t
    L.stencil_batch_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.stencil_batch_set_workspace.restype = st
    L.stencil_batch_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(stencil_info)]
    L.stencil_batch_info.restype = st
    L.stencil_batch_run.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i64, vp]
    L.stencil_batch_run.restype = st
    L.stencil_batch_run_graph.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i64, vp]
    L.stencil_batch_run_graph.restype = st
    L.stencil_batch_status.argtypes = [vp, vp]
    L.stencil_batch_status.restype = st
    L.stencil_batch_set_option.argtypes = [vp, ctypes.c_char_p, ctypes.c_char_p]
    L.stencil_batch_set_option.restype = st
    L.stencil_batch_destroy.argtypes = [vp]
    L.stencil_batch_autotune.argtypes = [vp, vp, vp, i64, ctypes.c_int, vp, ctypes.POINTER(stencil_batch_tune_result),
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.stencil_batch_autotune.restype = st
    L.stencil_batch_destroy.restype = None
    L.stencil_status_string.argtypes = [ctypes.c_int]
    L.stencil_status_string.restype = ctypes.c_char_p
    L.stencil_last_error.argtypes = []
    L.stencil_last_error.restype = ctypes.c_char_p
    L.stencil_launch_count.argtypes = []
    L.stencil_launch_count.restype = ctypes.c_uint64
    _LIB = L
    return L


def _check(status: int, what: str):
    if status != STENCIL_OK:
        msg = load().stencil_last_error().decode(errors="replace")
        raise StencilError(status, f"{what}: {msg}")


def _shape_code(shape) -> int:
    if isinstance(shape, str):
        return {"box": BOX, "star": STAR}[shape.lower()]
    return int(shape)


def _dtype_code(dtype) -> int:
    s = str(dtype)
    if s in ("f64", "float64", "torch.float64", "double", "0"):
        return F64
    if s in ("f32", "float32", "torch.float32", "float", "1"):
        return F32
    raise ValueError(f"dtype {dtype!r}: use f64 or f32")


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- C names ------------------------------------------------------------------

def stencil_plan_create(shape, d: int, r: int, weights, dtype, dims, t: int = 0) -> int:
    w = (ctypes.c_double * len(weights))(*[float(x) for x in weights])
    dd = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    h = ctypes.c_void_p()
    _check(load().stencil_plan_create(ctypes.byref(h), _shape_code(shape), int(d), int(r), w, _dtype_code(dtype), dd,
                                      int(t)), "stencil_plan_create")
    return h.value


def stencil_plan_set_option(plan: int, key: str, value) -> None:
    _check(load().stencil_plan_set_option(plan, key.encode(), str(value).encode()), f"stencil_plan_set_option({key})")


def stencil_plan_info(plan: int) -> dict:
    info = stencil_info()
    _check(load().stencil_plan_info(plan, ctypes.byref(info)), "stencil_plan_info")
    out = {f: getattr(info, f) for f, _ in stencil_info._fields_}
    out["tile"] = list(info.tile)
    out["path_name"] = PATH_NAMES[info.path]
    out["precision_name"] = PREC_NAMES[info.precision]
    return out


def stencil_plan_workspace_bytes(plan: int, for_host_io: bool = False) -> int:
    return int(load().stencil_plan_workspace_bytes(plan, 1 if for_host_io else 0))


def stencil_plan_set_workspace(plan: int, dev_ptr: int, nbytes: int) -> None:
    _check(load().stencil_plan_set_workspace(plan, dev_ptr, nbytes), "stencil_plan_set_workspace")


def stencil_run(plan: int, in_ptr: int, out_ptr: int, steps: int, stream=None) -> None:
    _check(load().stencil_run(plan, in_ptr, out_ptr, int(steps), _stream_handle(stream)), "stencil_run")


def stencil_run_noalloc(plan: int, in_ptr: int, out_ptr: int, steps: int, stream=None) -> None:
    _check(load().stencil_run_noalloc(plan, in_ptr, out_ptr, int(steps), _stream_handle(stream)),
           "stencil_run_noalloc")


def stencil_run_host(plan: int, host_in_ptr: int, host_out_ptr: int, steps: int, stream=None) -> None:
    _check(load().stencil_run_host(plan, host_in_ptr, host_out_ptr, int(steps), _stream_handle(stream)),
           "stencil_run_host")


def stencil_plan_tc_layout(plan: int, t: int, with_B: bool = True):
    """(layout dict, kb_lo list, kb_hi list, B array [a][kb][k][n] or None)."""
    import numpy as np
    lay = stencil_tc_layout()
    _check(load().stencil_plan_tc_layout(plan, int(t), ctypes.byref(lay), None, None, None), "stencil_plan_tc_layout")
    lines = 2 * lay.R + 1
    lo = (ctypes.c_int * lines)()
    hi = (ctypes.c_int * lines)()
    B = np.zeros((lines, lay.nkb, lay.k_inst, lay.n_tile), dtype=np.float64) if with_B else None
    _check(load().stencil_plan_tc_layout(plan, int(t), ctypes.byref(lay), lo, hi,
                                         B.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if with_B else None),
           "stencil_plan_tc_layout")
    d = {f: getattr(lay, f) for f, _ in stencil_tc_layout._fields_}
    return d, list(lo), list(hi), B


def stencil_device_status(stream=None) -> None:
    _check(load().stencil_device_status(_stream_handle(stream)), "stencil_device_status")


def stencil_plan_sptc_layout(plan: int, t: int):
    """Sparse (mma.sp TF32) operand layout: (layout dict, chunk_first, chunk_second,
    line_mask, values[lines, ns, 16, 8], select[lines, ns, 16, 8])."""
    import numpy as np
    lay = stencil_sptc_layout()
    _check(load().stencil_plan_sptc_layout(plan, t, ctypes.byref(lay), None, None, None, None, None),
           "stencil_plan_sptc_layout")
    lines, ns = 2 * lay.R + 1, lay.ns
    cf = np.zeros(2 * ns, np.int32)
    cs = np.zeros(2 * ns, np.int32)
    mask = np.zeros(lines, np.uint8)
    vals = np.zeros((lines, ns, 16, 8), np.float32)
    sel = np.zeros((lines, ns, 16, 8), np.uint8)
    _check(load().stencil_plan_sptc_layout(plan, t, ctypes.byref(lay), cf.ctypes.data, cs.ctypes.data,
                                           mask.ctypes.data, vals.ctypes.data, sel.ctypes.data),
           "stencil_plan_sptc_layout")
    d = {k: getattr(lay, k) for k, _ in stencil_sptc_layout._fields_}
    return d, cf, cs, mask, vals, sel


def stencil_plan_autotune(plan: int, in_ptr: int, out_ptr: int, steps: int, reps: int = 2, stream=None,
                          max_results: int = 64) -> list:
    res = (stencil_tune_result * max_results)()
    n = ctypes.c_int(0)
    _check(load().stencil_plan_autotune(plan, in_ptr, out_ptr, int(steps), int(reps), _stream_handle(stream), res,
                                        max_results, ctypes.byref(n)), "stencil_plan_autotune")
    return [{"path": PATH_NAMES[r.path], "precision": PREC_NAMES[r.precision], "t": r.t,
             "model_gstencils": r.model_gstencils, "measured_gstencils": r.measured_gstencils,
             "tile": (r.tile_y, r.tile_x)}
            for r in res[:min(n.value, max_results)]]


def stencil_plan_destroy(plan: int) -> None:
    if plan:
        load().stencil_plan_destroy(plan)


def stencil_model_predict(shape, d, r, t, dtype_bytes, sparsity, beta, P_cu, P_tc, B) -> dict:
    q = stencil_model_in(_shape_code(shape), d, r, t, dtype_bytes, sparsity, beta, P_cu, P_tc, B)
    o = stencil_model_out()
    _check(load().stencil_model_predict(ctypes.byref(q), ctypes.byref(o)), "stencil_model_predict")
    return {f: getattr(o, f) for f, _ in stencil_model_out._fields_}


def stencil_set_peaks(**kw) -> None:
    p = stencil_peaks(**kw)
    _check(load().stencil_set_peaks(ctypes.byref(p)), "stencil_set_peaks")


def stencil_get_peaks() -> dict:
    p = stencil_peaks()
    _check(load().stencil_get_peaks(ctypes.byref(p)), "stencil_get_peaks")
    return {f: getattr(p, f) for f, _ in stencil_peaks._fields_}


def stencil_probe_peaks(stream=None) -> dict:
    p = stencil_peaks()
    _check(load().stencil_probe_peaks(ctypes.byref(p), _stream_handle(stream)), "stencil_probe_peaks")
    return {f: getattr(p, f) for f, _ in stencil_peaks._fields_}


def stencil_status_string(s: int) -> str:
    return load().stencil_status_string(s).decode()


def stencil_last_error() -> str:
    return load().stencil_last_error().decode(errors="replace")


def stencil_launch_count() -> int:
    return int(load().stencil_launch_count())


def declared_symbols(header: str | None = None) -> list[str]:
    """Function names declared in include/gbstencil.h."""
    header = header or os.path.join(_build.INCLUDE, "gbstencil.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stencil_[a-z0-9_]+)\s*\(", text)))


# ---- convenience wrapper over torch tensors ----------------------------------------

def stencil_host_alloc(nbytes: int) -> int:
    p = ctypes.c_void_p()
    _check(load().stencil_host_alloc(ctypes.byref(p), int(nbytes)), "stencil_host_alloc")
    return p.value


def stencil_host_free(ptr: int) -> None:
    _check(load().stencil_host_free(ptr), "stencil_host_free")


def host_empty(shape, dtype):
    """A CPU torch tensor of `shape` and `dtype` ("f64"/"f32") in memory from
    stencil_host_alloc (huge-page backed, page-locked); the memory is released
    with the tensor."""
    import numpy as np
    import torch
    npdt = np.float64 if _dtype_code(dtype) == F64 else np.float32
    count = 1
    for n in shape:
        count *= int(n)
    nbytes = max(count, 1) * np.dtype(npdt).itemsize
    ptr = stencil_host_alloc(nbytes)
    arr = np.ctypeslib.as_array((ctypes.c_char * nbytes).from_address(ptr)).view(npdt)[:count].reshape(shape)
    t = torch.from_numpy(arr)
    import weakref
    weakref.finalize(t, stencil_host_free, ptr)
    return t


def _resolve_device(device):
    """torch.device with the index filled in ("cuda" -> the current CUDA
    device), so that it compares equal to the device of a tensor on it."""
    import torch
    dev = torch.device(device)
    if dev.type == "cuda" and dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    return dev


class Plan:
    """A plan plus PyTorch-allocated workspace.  run() takes CUDA tensors of
    the stored shape (interior + 2r per axis) and the plan's dtype."""

    def __init__(self, shape, d, r, weights, dtype, dims, t: int = 0, **options):
        self.shape, self.d, self.r = shape, int(d), int(r)
        self.dims = tuple(int(x) for x in dims)
        self.dtype = "f64" if _dtype_code(dtype) == F64 else "f32"
        self.handle = stencil_plan_create(shape, d, r, weights, dtype, dims, t)
        self._ws = None
        for k, v in options.items():
            stencil_plan_set_option(self.handle, k, v)

    @property
    def stored_shape(self):
        return tuple(n + 2 * self.r for n in self.dims)

    def set_option(self, key, value):
        stencil_plan_set_option(self.handle, key, value)

    def info(self) -> dict:
        return stencil_plan_info(self.handle)

    def _torch_dtype(self):
        import torch
        return torch.float64 if self.dtype == "f64" else torch.float32

    def ensure_workspace(self, device, host_io: bool = False):
        import torch
        device = _resolve_device(device)
        need = stencil_plan_workspace_bytes(self.handle, host_io)
        if self._ws is None or self._ws.numel() < need or self._ws.device != device:
            self._ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
            stencil_plan_set_workspace(self.handle, self._ws.data_ptr(), self._ws.numel())
        return self._ws

    def _check_tensor(self, x, name):
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if x.dtype != self._torch_dtype() or not x.is_contiguous() or tuple(x.shape) != self.stored_shape:
            raise ValueError(f"{name}: need a contiguous {self._torch_dtype()} tensor of shape {self.stored_shape}")

    def run(self, x_in, x_out, steps: int, stream=None):
        self._check_tensor(x_in, "in")
        self._check_tensor(x_out, "out")
        self.ensure_workspace(x_in.device)
        stencil_run(self.handle, x_in.data_ptr(), x_out.data_ptr(), steps, stream)

    def autotune(self, x_in, x_out, steps: int, reps: int = 2, stream=None) -> list:
        self._check_tensor(x_in, "in")
        self._check_tensor(x_out, "out")
        self.ensure_workspace(x_in.device)
        return stencil_plan_autotune(self.handle, x_in.data_ptr(), x_out.data_ptr(), steps, reps, stream)

    def run_host(self, h_in, h_out, steps: int, device="cuda", stream=None):
        """h_in/h_out: CPU tensors (pinned for full speed) of the stored shape."""
        import torch
        for x, n in ((h_in, "host in"), (h_out, "host out")):
            if not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != self._torch_dtype() \
                    or not x.is_contiguous() or tuple(x.shape) != self.stored_shape:
                raise ValueError(f"{n}: need a contiguous CPU {self._torch_dtype()} tensor of shape "
                                 f"{self.stored_shape}")
        self.ensure_workspace(device, host_io=True)
        stencil_run_host(self.handle, h_in.data_ptr(), h_out.data_ptr(), steps, stream)

    def close(self):
        if getattr(self, "handle", None):
            stencil_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched form ---------------------------------------------------------------

def stencil_batch_create(grids, dtype, t: int = 0) -> int:
    """grids: iterable of (shape, r, ny, nx, weights)."""
    grids = list(grids)
    keep = []
    arr = (stencil_grid_desc * len(grids))()
    for i, (shape, r, ny, nx, w) in enumerate(grids):
        wa = (ctypes.c_double * len(w))(*[float(x) for x in w])
        keep.append(wa)
        arr[i] = stencil_grid_desc(_shape_code(shape), int(r), int(ny), int(nx),
                                   ctypes.cast(wa, ctypes.POINTER(ctypes.c_double)))
    h = ctypes.c_void_p()
    _check(load().stencil_batch_create(ctypes.byref(h), len(grids), arr, _dtype_code(dtype), int(t)),
           "stencil_batch_create")
    return h.value


def stencil_batch_workspace_bytes(batch: int, steps: int) -> int:
    return int(load().stencil_batch_workspace_bytes(batch, int(steps)))


def stencil_batch_set_workspace(batch: int, dev_ptr: int, nbytes: int) -> None:
    _check(load().stencil_batch_set_workspace(batch, dev_ptr, nbytes), "stencil_batch_set_workspace")


def stencil_batch_info(batch: int, i: int) -> dict:
    info = stencil_info()
    _check(load().stencil_batch_info(batch, int(i), ctypes.byref(info)), "stencil_batch_info")
    out = {f: getattr(info, f) for f, _ in stencil_info._fields_}
    out["tile"] = list(info.tile)
    return out


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[int(p) for p in ptrs])


def stencil_batch_run(batch: int, in_ptrs, out_ptrs, steps: int, stream=None) -> None:
    _check(load().stencil_batch_run(batch, _ptr_array(in_ptrs), _ptr_array(out_ptrs), int(steps),
                                    _stream_handle(stream)), "stencil_batch_run")


def stencil_batch_run_graph(batch: int, in_ptrs, out_ptrs, steps: int, stream=None) -> None:
    _check(load().stencil_batch_run_graph(batch, _ptr_array(in_ptrs), _ptr_array(out_ptrs), int(steps),
                                          _stream_handle(stream)), "stencil_batch_run_graph")


def stencil_batch_status(batch: int, stream=None) -> None:
    _check(load().stencil_batch_status(batch, _stream_handle(stream)), "stencil_batch_status")


def stencil_batch_set_option(batch: int, key: str, value) -> None:
    _check(load().stencil_batch_set_option(batch, key.encode(), str(value).encode()),
           f"stencil_batch_set_option({key})")


def stencil_batch_autotune(batch: int, in_ptrs, out_ptrs, steps: int, reps: int = 1, stream=None,
                           max_results: int = 2048) -> list:
    res = (stencil_batch_tune_result * max_results)()
    n = ctypes.c_int(0)
    _check(load().stencil_batch_autotune(batch, _ptr_array(in_ptrs), _ptr_array(out_ptrs), int(steps), int(reps),
                                         _stream_handle(stream), res, max_results, ctypes.byref(n)),
           "stencil_batch_autotune")
    out = []
    for q in res[:min(n.value, max_results)]:
        d = {f: getattr(q, f) for f, _ in stencil_batch_tune_result._fields_}
        d["shape"] = "box" if q.shape == 0 else "star"
        d["path"] = PATH_NAMES[q.path]
        d["precision"] = PREC_NAMES[q.precision]
        d["chosen"] = bool(q.chosen)
        out.append(d)
    return out


def stencil_batch_destroy(batch: int) -> None:
    if batch:
        load().stencil_batch_destroy(batch)


class Batch:
    """A batch of 2-D grids with PyTorch-allocated workspace."""

    def __init__(self, grids, dtype, t: int = 0):
        self.grids = [(g[0], int(g[1]), int(g[2]), int(g[3]), g[4]) for g in grids]
        self.dtype = "f64" if _dtype_code(dtype) == F64 else "f32"
        self.handle = stencil_batch_create(self.grids, dtype, t)
        self._ws = None
        self._ws_steps = None

    def stored_shape(self, i):
        _, r, ny, nx, _ = self.grids[i]
        return (ny + 2 * r, nx + 2 * r)

    def info(self, i):
        return stencil_batch_info(self.handle, i)

    def ensure_workspace(self, steps, device="cuda"):
        import torch
        device = _resolve_device(device)
        need = stencil_batch_workspace_bytes(self.handle, steps)
        if self._ws is None or self._ws.numel() < need or self._ws.device != device:
            self._ws = torch.empty(max(need, 1), dtype=torch.uint8, device=device)
            stencil_batch_set_workspace(self.handle, self._ws.data_ptr(), self._ws.numel())
        return self._ws

    def set_option(self, key, value):
        stencil_batch_set_option(self.handle, key, value)

    def autotune(self, ins, outs, steps: int, reps: int = 1, stream=None) -> list:
        """Tune (path, t, tile) per shape class on these buffers (outputs are
        overwritten); the next run re-sizes the workspace if it must."""
        self.ensure_workspace(steps, ins[0].device)
        return stencil_batch_autotune(self.handle, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs], steps,
                                      reps, stream)

    def run(self, ins, outs, steps: int, stream=None, graph: bool = False):
        self.ensure_workspace(steps, ins[0].device)
        fn = stencil_batch_run_graph if graph else stencil_batch_run
        fn(self.handle, [x.data_ptr() for x in ins], [y.data_ptr() for y in outs], steps, stream)

    def close(self):
        if getattr(self, "handle", None):
            stencil_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
