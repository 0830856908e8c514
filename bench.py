#!/usr/bin/env python3
"""GStencil/s of the GB300 stencil engine on the Box-2D3R FP64 16384^2 workload.

One bench step = one call of stencil_run over the whole workload (100 steps
of Box-2D3R FP64 on a 16384 x 16384 interior with a fixed zero halo of width
3), i.e. every fused sweep of the dispatched plan plus the halo copy.  The
plan (path and fusion depth t) is what the library's model-based dispatcher
picks; `--t` / `--path` force one.  Inputs are seeded synthetic data of the
paper's kind (weights U(0,1) normalised to sum 1, field U[0,1)).

Printed: one JSON line (rank 0).  value = point-updates per second / 1e9
summed over ranks (each rank runs its own replica: weak scaling), timed with
CUDA events between barriers, inputs resident in HBM and larger than L2.
e2e = the same metric through stencil_run_host (pinned host buffers, copies
inside the timed region).  roofline = the dominant kernel (the sweep)
against the FP64 FMA pipe (ALU-bound) or HBM (memory-bound configurations).
cpu_baseline = the CPU oracle on a bounded sample of the same workload.

--impl reference times the CPU oracle alone (the comparison arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GStencil/s and % of roofline, mixed-precision & batched vs plain FP64, 1 GB300"
UNIT = "GStencil/s"

WORKLOADS = {
    # name: shape, d, r, interior dims, steps per run, dtype, seed
    "box2d3r_f64_16384": dict(shape="box", d=2, r=3, dims=(16384, 16384), steps=100, dtype="f64", seed=2),
    "star2d1r_f64_512": dict(shape="star", d=2, r=1, dims=(512, 512), steps=10, dtype="f64", seed=1),
    "star3d2r_f64_512": dict(shape="star", d=3, r=2, dims=(512, 512, 512), steps=50, dtype="f64", seed=3),
    "star3d2r_f32_512": dict(shape="star", d=3, r=2, dims=(512, 512, 512), steps=50, dtype="f32", seed=3),
    "box3d1r_f64_512": dict(shape="box", d=3, r=1, dims=(512, 512, 512), steps=50, dtype="f64", seed=3),
    "box3d1r_f32_512": dict(shape="box", d=3, r=1, dims=(512, 512, 512), steps=50, dtype="f32", seed=3),
    "box2d2r_f32_16384": dict(shape="box", d=2, r=2, dims=(16384, 16384), steps=1000, dtype="f32", seed=4,
                              field="sine"),
}
DEFAULT = "box2d3r_f64_16384"

# Derived ALU peaks (152 SMs x 2070 MHz maximum clock; per SM and clock: 2 FP64
# FMA lanes = 4 FLOP, 128 FP32 FMA lanes = 256 FLOP).
SMS, SM_MAX_MHZ = 152, 2070.0
ALU_PEAK_TFLOPS = {"f64": SMS * SM_MAX_MHZ * 1e6 * 4 / 1e12, "f32": SMS * SM_MAX_MHZ * 1e6 * 256 / 1e12}
FALLBACK_HBM_GBS = 6800.0


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def points_of(cfg):
    return math.prod(cfg["dims"])


def config_json(name, cfg, extra=None):
    c = {"workload": f"{cfg['shape'].capitalize()}-{cfg['d']}D{cfg['r']}R {cfg['dtype'].upper()} "
                     f"{'x'.join(str(n) for n in cfg['dims'])}, {cfg['steps']} steps",
         "name": name, "shape": cfg["shape"], "d": cfg["d"], "r": cfg["r"],
         "dims": list(cfg["dims"]), "steps_per_run": cfg["steps"], "halo": "fixed zeros, width r",
         "l2": "inputs larger than L2 (no flush)" if points_of(cfg) * (8 if cfg["dtype"] == "f64" else 4) > 129e6
         else "inputs smaller than L2"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------------------
# clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return None
        self.file.flush()
        with open(self.file.name) as f:
            rows = [[c.strip() for c in line.split(",")] for line in f if line.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
def cpu_baseline(cfg, w, u, budget_s=15.0):
    """The oracle (as it stands) on a bounded sample of the workload: the same
    grid and initial field, but only as many of its steps as take about
    budget_s of CPU time (at least one)."""
    import numpy as np

    import oracle
    u64 = np.ascontiguousarray(u, dtype=np.float64)
    d = cfg["d"]
    t0 = time.perf_counter()
    oracle.run(cfg["shape"], d, cfg["r"], w, cfg["dims"], u64, 1)  # calibration: one step of the full grid
    one = time.perf_counter() - t0
    steps = max(1, min(cfg["steps"], int(budget_s / max(one, 1e-9))))
    t0 = time.perf_counter()
    oracle.run(cfg["shape"], d, cfg["r"], w, cfg["dims"], u64, steps)
    el = time.perf_counter() - t0
    return {"value": points_of(cfg) * steps / el / 1e9, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": f"the full {'x'.join(map(str, cfg['dims']))} grid for {steps} of its {cfg['steps']} steps, "
                      f"FP64 C oracle with OpenMP ({el:.1f} s)"}


def run_reference(args, cfg, name, rank):
    """Comparison arm: the CPU oracle on the machine's host cores."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2603_00477_gb300 import inputs
    oracle.build()
    d = cfg["d"]
    side = 1024 if d == 2 else 96
    dims = (side,) * d
    npdt = np.float64 if cfg["dtype"] == "f64" else np.float32
    w, u = inputs.problem(cfg["shape"], d, cfg["r"], dims, seed=cfg["seed"], dtype=npdt)
    u = u.astype(np.float64)
    t0 = time.perf_counter()
    oracle.run(cfg["shape"], d, cfg["r"], w, dims, u, 1)
    one = time.perf_counter() - t0
    per_step_budget = min(8.0, 150.0 / max(1, args.steps + args.warmup))
    sample_steps = max(1, min(cfg["steps"], int(per_step_budget / max(one, 1e-6))))
    for _ in range(args.warmup):
        oracle.run(cfg["shape"], d, cfg["r"], w, dims, u, sample_steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(cfg["shape"], d, cfg["r"], w, dims, u, sample_steps)
    el = time.perf_counter() - t0
    value = math.prod(dims) * sample_steps * args.steps / el / 1e9
    sample = (f"{cfg['shape']}-{d}D{cfg['r']}R {cfg['dtype']} on a {'x'.join(map(str, dims))} interior, "
              f"{sample_steps} steps per bench step, FP64 C oracle with OpenMP")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded splitmix64)",
            "config": config_json(name, cfg, {"sample": sample}), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def traffic_record(kernel_key):
    """DRAM bytes per launch of `kernel_key` from the committed ncu summary, if
    the kernel source has not changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic_per_launch.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(kernel_key)
    if not rec:
        return None
    h = hashlib.sha256()
    for src in rec.get("sources", []):
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return float(rec["dram_bytes_per_launch"])



def kernel_name(info: dict, d: int, dtype: str, shape: str = "box", r: int = 1) -> str:
    """The sweep kernel a plan launches, from its stencil, path, precision,
    tile and t (the rules of the library's launchers)."""
    if info["path"] == 1:
        if d == 2:
            return "cu2d_sweep"
        if info["t"] != 1:
            return "cu3d_sweep"
        # FP32 star r <= 3 and box r = 1 take the rotating kernel
        rot = dtype == "f32" and ((shape == "star" and r <= 3) or (shape == "box" and r == 1))
        return "cu3d_rot" if rot else "cu3d_stream"
    if info["path"] == 3:
        return "sptc2d_sweep"
    if d == 3:
        return "tc3d_wide"
    if dtype == "f64":
        return "tc2d_split" if info["precision_name"] == "ozaki" else "dmma2d_sweep"
    if info["precision_name"] in ("f16", "f16x3", "bf16x3"):
        return "tc2d_wide"
    return "tc2d_ws"


def max_over_ranks(x: float, world: int) -> float:
    """The largest per-rank value (a duration): every rank gets the maximum.
    Uses a CUDA tensor under NCCL and a CPU tensor under gloo."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world: int, points: int, steps_per_run: int, runs: int, seconds: float) -> float:
    """Point-updates per second / 1e9 over all ranks: each rank runs its own
    replica (weak scaling), the job takes the slowest rank's time."""
    return world * points * steps_per_run * runs / seconds / 1e9


def _time_runs(fn, stream, reps=3, warm=1):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


# The stencils of the paper's problem classification (2-D and 3-D, radius 1 and
# 2) plus the radii its benchmarks use (3 and 7 in 2-D), box and star.
CLASSIFY_STENCILS = [(s, 2, r) for s in ("box", "star") for r in (1, 2, 3, 7)] + \
                    [(s, 3, r) for s in ("box", "star") for r in (1, 2)]
# The paper's six representative cases (Sec. 5: stencil, t, element type,
# tensor-core form), re-evaluated with this engine's tiles.
PAPER_CASES = [("box", 2, 1, 3, "f64", "tensor_core", None), ("box", 2, 3, 1, "f64", "tensor_core", None),
               ("box", 2, 1, 7, "f32", "sparse_tensor_core", "tf32"),
               ("box", 2, 7, 1, "f32", "sparse_tensor_core", "tf32"),
               ("box", 3, 1, 3, "f64", "tensor_core", None), ("box", 3, 1, 7, "f32", "sparse_tensor_core", "tf32")]


def _stencil_name(shape, d, r):
    return f"{shape.capitalize()}-{d}D{r}R"


def model_leg(B, inputs, tmax=8):
    """The model of Secs. 3-4 evaluated on this GPU's peaks, host only.

    classification: for FP32 and FP64 and every stencil of CLASSIFY_STENCILS,
    the CUDA-core intensity I^(t) of Eq. 8 for t = 1..tmax against the FP
    pipe's ridge point, and the first t at which the stencil becomes compute
    bound (the paper's problem-classification figure, which shows FP32 on an
    A100).  cases: the paper's six representative cases with the CUDA-core
    plan and the tensor-core plan this engine would run (its alpha, its tiles'
    S, Eq. 12 intensity, ridge, scenario and predicted rates); null where no
    tensor-core kernel covers the case (3-D)."""
    peaks = B.stencil_get_peaks()
    out = {"peaks": peaks, "tmax": tmax, "classification": {}, "cases": []}
    for dtype, D, P in (("f32", 4, peaks["cu_f32_flops"]), ("f64", 8, peaks["cu_f64_flops"])):
        rows = []
        for shape, d, r in CLASSIFY_STENCILS:
            I, bound = [], []
            for t in range(1, tmax + 1):
                m = B.stencil_model_predict(shape, d, r, t, D, 1.0, 1.0, P, P, peaks["hbm_bytes_per_s"])
                I.append(m["I_cu"])
                bound.append("compute" if m["I_cu"] >= m["ridge_cu"] else "memory")
            first = next((t for t, b in enumerate(bound, 1) if b == "compute"), None)
            rows.append({"stencil": _stencil_name(shape, d, r), "I": I, "bound": bound,
                         "ridge": P / peaks["hbm_bytes_per_s"], "compute_bound_from_t": first})
        out["classification"][dtype] = rows
    keys = ("t", "alpha", "sparsity", "beta", "intensity", "ridge", "scenario", "memory_bound",
            "predicted_gstencils", "path_name", "precision_name")
    for shape, d, r, t, dtype, tc_path, prec in PAPER_CASES:
        dims = (10240, 10240) if d == 2 else (1024, 1024, 1024)
        w = inputs.weights(shape, d, r, 1)
        case = {"stencil": _stencil_name(shape, d, r), "t": t, "dtype": dtype, "dims": list(dims)}
        cu = B.Plan(shape, d, r, w, dtype, dims, t)
        cu.set_option("path", "cuda_core")
        ci = cu.info()
        case["cuda_core"] = {k: ci[k] for k in keys}
        case["cuda_core"]["roof_gstencils"] = ci["predicted_cu_gstencils"]
        cu.close()
        try:
            tc = B.Plan(shape, d, r, w, dtype, dims, t)
            if prec:
                tc.set_option("precision", prec)
            tc.set_option("path", tc_path)
            ti = tc.info()
            case["tensor_core"] = {k: ti[k] for k in keys}
            case["scenario"] = ti["scenario"]
            tc.close()
        except B.StencilError as e:
            case["tensor_core"] = None
            case["tensor_core_unavailable"] = str(e)
            case["scenario"] = ci["scenario"]
        out["cases"].append(case)
    return out


def fusion_leg(B, inputs, stream, dims=(4096, 4096), tmax=8):
    """The paper's intensity-versus-fusion-depth measurement (Sec. 5.2, the
    figure of measured I against t), on this engine's FP64 CUDA-core sweep:
    for Box-2D1R and Star-2D1R and t = 1..tmax, one fused sweep of depth t over
    a grid larger than L2, timed with CUDA events, next to the model's
    intensity I = tK/D (Eq. 8) and predicted rate.  Each (stencil, t) launches
    the sweep kernel twice (an untimed warm-up, then the timed launch), so an
    ncu capture of the kernel sees 2 * 2 * tmax launches in this order; its
    DRAM bytes and FP64 instruction counts give the measured C, M and I."""
    import numpy as np
    import torch
    rows = []
    for shape in ("box", "star"):
        w, u = inputs.problem(shape, 2, 1, dims, seed=21, dtype=np.float64)
        x = torch.from_numpy(u).cuda()
        y = torch.empty_like(x)
        for t in range(1, tmax + 1):
            plan = B.Plan(shape, 2, 1, w, "f64", dims, t)
            plan.set_option("path", "cuda_core")
            info = plan.info()
            sec = _time_runs(lambda: plan.run(x, y, t), stream, reps=1, warm=1)
            rows.append({"stencil": _stencil_name(shape, 2, 1), "t": t, "K": info["K"],
                         "tile": info["tile"], "gstencils": math.prod(dims) * t / sec / 1e9,
                         "sweep_ms": sec * 1e3, "model_intensity": info["intensity"],
                         "model_gstencils": info["predicted_gstencils"],
                         "model_memory_bound": bool(info["memory_bound"])})
            plan.close()
        del x, y
        torch.cuda.empty_cache()
    return {"workload": f"FP64 {'x'.join(map(str, dims))}, one fused sweep of depth t per row", "rows": rows}


def mixed_precision_leg(B, inputs, stream, steps=100, horizon=1000, every=100, fine=10):
    """Box-2D2R FP32 16384^2 (sine-mode field): plain FP32 on CUDA cores
    against the tensor-core TF32, TF32x3, BF16x3, F16 and F16x3 forms and the
    sparse TF32 form at each t = 1..4 (point-updates/s over `steps`-step
    runs), then, for plain FP32 and each form at its fastest t, the normwise
    relative error every `fine` steps up to `every` steps and every `every`
    steps up to `horizon` steps against the FP64 CUDA-core path run on the GPU
    from the same field (the reference the GPU tests hold within 1e-12 of the
    FP64 oracle); then the same field stored in FP64: plain FP64 on CUDA cores
    against FP64 by exact splitting on the FP16 tensor cores (rates, and the
    split form's error every `every` steps to `horizon`)."""
    import numpy as np
    import torch
    dims = (16384, 16384)
    w, u = inputs.problem("box", 2, 2, dims, seed=4, dtype=np.float32, field="sine")
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    pts = dims[0] * dims[1]
    rows = []
    cands = [("cuda_core", "native", t) for t in (1, 2, 3, 4)] + \
            [("tensor_core", p, t) for p in ("tf32", "tf32x3", "bf16x3", "f16", "f16x3") for t in (1, 2, 3, 4)] + \
            [("sparse_tensor_core", "tf32", t) for t in (1, 2, 3, 4)]
    for path, prec, t in cands:
        plan = B.Plan("box", 2, 2, w, "f32", dims, t)
        if prec != "native":
            plan.set_option("precision", prec)
        plan.set_option("path", path)
        plan.ensure_workspace(x.device)
        sec = _time_runs(lambda: plan.run(x, y, steps), stream)
        info = plan.info()
        rows.append({"path": path, "precision": prec, "t": t, "gstencils": pts * steps / sec / 1e9,
                     "model_gstencils": info["predicted_gstencils"], "alpha": info["alpha"],
                     "sparsity": info["sparsity"], "beta": info["beta"]})
        plan.close()
    plain = max(r["gstencils"] for r in rows if r["path"] == "cuda_core")
    best = max(rows, key=lambda r: r["gstencils"])
    # CUDA cores vs tensor cores at each t: the model's winner and the measured one
    crossover = []
    for t in (1, 2, 3, 4):
        at = [r for r in rows if r["t"] == t and r["precision"] in ("native", "tf32")]
        m = max(at, key=lambda r: r["model_gstencils"])
        g = max(at, key=lambda r: r["gstencils"])
        crossover.append({"t": t, "model_winner": m["path"], "measured_winner": g["path"],
                          "cuda_core_gstencils": next(r["gstencils"] for r in at if r["path"] == "cuda_core"),
                          "best_tensor_gstencils": max(r["gstencils"] for r in at if r["path"] != "cuda_core")})
    # the same over every form (FP16 has TF32's normwise error; the 3-product
    # forms are more accurate)
    crossover_all = []
    for t in (1, 2, 3, 4):
        at = [r for r in rows if r["t"] == t]
        m = max(at, key=lambda r: r["model_gstencils"])
        g = max(at, key=lambda r: r["gstencils"])
        crossover_all.append({"t": t, "model_winner": f'{m["path"]}:{m["precision"]}',
                              "measured_winner": f'{g["path"]}:{g["precision"]}',
                              "measured_best_gstencils": g["gstencils"]})

    # error growth: FP64 reference states every `fine` steps to `every`, then
    # every `every` steps (kept on the GPU)
    marks = list(range(fine, every, fine)) + list(range(every, horizon + 1, every))
    ref_plan = B.Plan("box", 2, 2, w, "f64", dims, 0)
    ref_plan.set_option("path", "cuda_core")
    a64 = x.double()
    b64 = torch.empty_like(a64)
    ref_plan.ensure_workspace(a64.device)
    refs = []
    done_steps = 0
    for m in marks:
        ref_plan.run(a64, b64, m - done_steps)
        done_steps = m
        refs.append(b64[2:-2, 2:-2].clone())
        a64, b64 = b64, a64
    ref_plan.close()
    del a64, b64
    errors = []
    fastest = {}
    for r in rows:
        k = (r["path"], r["precision"])
        if k not in fastest or r["gstencils"] > fastest[k]["gstencils"]:
            fastest[k] = r
    for (path, prec), r in fastest.items():
        plan = B.Plan("box", 2, 2, w, "f32", dims, r["t"])
        if prec != "native":
            plan.set_option("precision", prec)
        plan.set_option("path", path)
        plan.ensure_workspace(x.device)
        a, b = x.clone(), torch.empty_like(x)
        curve = []
        done_steps = 0
        for m, ref in zip(marks, refs):
            plan.run(a, b, m - done_steps)  # runs restart the fused schedule at each mark
            done_steps = m
            d = (b[2:-2, 2:-2].double() - ref).abs().max() / ref.abs().max()
            curve.append({"steps": m, "rel_linf": float(d)})
            a, b = b, a
        plan.close()
        del a, b
        held = 0
        for c in curve:
            if c["rel_linf"] > 2e-6:
                break
            held = c["steps"]
        errors.append({"path": path, "precision": prec, "t": r["t"], "gstencils": r["gstencils"],
                       "error_vs_fp64": curve, "within_2e-6_up_to_steps": held})
    # the same field stored in FP64: plain FP64 on CUDA cores against the FP64
    # grid on the FP16 tensor cores by exact splitting (rate over `steps`
    # steps; error every `every` steps to `horizon` against the FP64 reference)
    ref_at = dict(zip(marks, refs))
    fp64_storage = []
    x64 = x.double()
    y64 = torch.empty_like(x64)
    for path, prec, t in (("cuda_core", "native", 1), ("tensor_core", "ozaki", 1), ("tensor_core", "ozaki", 2)):
        plan = B.Plan("box", 2, 2, w, "f64", dims, t)
        if prec != "native":
            plan.set_option("precision", prec)
        plan.set_option("path", path)
        plan.ensure_workspace(x64.device)
        sec = _time_runs(lambda: plan.run(x64, y64, steps), stream)
        row = {"path": path, "precision": prec, "t": t, "gstencils": pts * steps / sec / 1e9,
               "model_gstencils": plan.info()["predicted_gstencils"]}
        if prec != "native":
            a, b = x64.clone(), torch.empty_like(x64)
            curve = []
            for m in range(every, horizon + 1, every):
                plan.run(a, b, every)
                ref = ref_at[m]
                curve.append({"steps": m, "rel_linf": float((b[2:-2, 2:-2] - ref).abs().max() / ref.abs().max())})
                a, b = b, a
            del a, b
            row["error_vs_fp64"] = curve
            row["within_2e-6_up_to_steps"] = horizon if all(c["rel_linf"] <= 2e-6 for c in curve) else None
        plan.close()
        fp64_storage.append(row)
    del x64, y64, ref_at
    del refs, x, y
    torch.cuda.empty_cache()
    return {"workload": f"Box-2D2R F32 16384x16384, sine-mode field, {steps} steps per timed run; "
                        f"error every {every} steps to {horizon}",
            "error_reference": "FP64 CUDA-core path on the GPU (held within 1e-12 of the FP64 oracle by the GPU tests, "
                               "16384^2 x 100 steps on sampled boxes included)",
            "plain_fp32_cuda_core_gstencils": plain, "best": best, "crossover": crossover,
            "crossover_all_forms": crossover_all, "rows": rows,
            "errors": errors, "fp64_storage": fp64_storage}


def split_fp64_leg(B, cfg, w, x, y_plain, plain_gstencils, stream, reps):
    """FP64 on the FP16 tensor cores by exact splitting (precision "ozaki")
    on the headline FP64 workload, next to the plain FP64 path already timed:
    point-updates/s over `reps` runs (CUDA events), the normwise error against
    the plain path's result on the whole grid (the GPU tests hold both paths
    within 1e-12 of the oracle, on this grid and step count on sampled boxes),
    and the tensor-core work of its kernel (tc2d_split):
    useful FP64 FLOP (2K per point-step) and issued FP16 MMA FLOP (the model's
    beta/S times the useful work, beta = S(S+1)/2 digit products)."""
    import torch

    dims, steps = cfg["dims"], cfg["steps"]
    if cfg["d"] != 2:
        return None
    plan = B.Plan(cfg["shape"], 2, cfg["r"], w, "f64", dims, 0)
    try:
        plan.set_option("precision", "ozaki")
        plan.set_option("path", "tensor_core")
    except B.StencilError as e:
        plan.close()
        return {"unavailable": str(e)}
    info = plan.info()
    plan.ensure_workspace(x.device)
    z = torch.empty_like(x)
    sec = _time_runs(lambda: plan.run(x, z, steps), stream, reps=reps, warm=1)
    pts = math.prod(dims)
    value = pts * steps / sec / 1e9
    r = cfg["r"]
    inner = (slice(r, -r), slice(r, -r))
    err_plain = float((z[inner] - y_plain[inner]).abs().max() / y_plain[inner].abs().max())
    t = info["t"]
    nsweeps = steps // t + (1 if steps % t else 0)
    launch_s = sec / nsweeps
    useful = pts * 2 * info["K"] * (steps / nsweeps)  # FLOP of one sweep (t steps)
    issued = useful * info["alpha"] * info["beta"] / info["sparsity"]
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 0.0)) or 0.0)
    S = int(round((math.sqrt(1 + 8 * info["beta"]) - 1) / 2))
    plan.close()
    del z
    torch.cuda.empty_cache()
    return {"workload": config_json("", cfg)["workload"], "path": "tensor_core", "precision": "ozaki",
            "t": t, "digit_slices": S, "products_per_useful_product": info["beta"], "sparsity": info["sparsity"],
            "gstencils": value, "vs_plain_fp64": value / plain_gstencils if plain_gstencils else None,
            "model_gstencils": info["predicted_gstencils"],
            "rel_linf_vs_plain_fp64_gpu": err_plain,
            "kernel": {"name": "tc2d_split", "avg_launch_ms": launch_s * 1e3,
                       "useful_fp64_tflops": useful / launch_s / 1e12,
                       "issued_fp16_tflops": issued / launch_s / 1e12, "peak_tflops": peak,
                       "peak_source": f"bf16_tflops_sustained of {src} peaks (FP16 and BF16 share the dense rate)",
                       "issued_frac": issued / launch_s / 1e12 / peak if peak else None}}


def table3_leg(B, inputs, stream):
    """The paper's six representative cases (Table 3, Sec. 5.3) measured on
    GB300 at the paper's domain sizes (Sec. 5.1: 10240^2 in 2-D, 1024^3 in
    3-D): each case's CUDA-core form and, in 2-D, its tensor-core form (the
    FP64 MMA for FP64 cases, 2:4-sparse TF32 for FP32 ones) at the case's t,
    with the model's prediction and scenario for both, the measured
    direction of change (tensor-core rate / CUDA-core rate) next to the
    paper's A100 one, and this engine's fastest tensor-core form for the
    case (FP64 by exact splitting; FP16 with the operands exchanged).  The
    3-D cases are fused (t = 3, 7), which the 3-D tensor-core kernel (t = 1)
    does not cover: they run on CUDA cores at the case's t and at t = 1, and
    the FP32 case also in the 3-D FP16 tensor-core form at t = 1."""
    import numpy as np
    import torch
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_table3.json")))
    out = []
    for case in gold["cases"]:
        shape, d, r, t, D = case["shape"], case["d"], case["r"], case["t"], case["D"]
        dtype = "f64" if D == 8 else "f32"
        dims = (10240, 10240) if d == 2 else (1024, 1024, 1024)
        steps = 3 * t if d == 2 else t
        w, u = inputs.problem(shape, d, r, dims, seed=case["case"], dtype=np.float64 if D == 8 else np.float32)
        x = torch.from_numpy(u).cuda()
        del u
        y = torch.empty_like(x)
        pts = math.prod(dims)
        forms = [("cuda_core", None, t)]
        if d == 2:
            forms.append(("sparse_tensor_core", "tf32", t) if case["tc"] == "sptc_tf32" else ("tensor_core", "native", t))
            forms.append(("tensor_core", "ozaki" if D == 8 else "f16", t))
        else:
            if t != 1:
                forms.append(("cuda_core", None, 1))
            if D == 4:
                forms.append(("tensor_core", "f16", 1))
        res = {"case": case["case"], "stencil": f"{shape.capitalize()}-{d}D{r}R", "t": t, "dtype": dtype,
               "dims": list(dims), "steps_per_run": steps, "paper_change_a100": case["change"], "forms": []}
        for path, prec, tt in forms:
            try:
                plan = B.Plan(shape, d, r, w, dtype, dims, tt)
                if prec:
                    plan.set_option("precision", prec)
                plan.set_option("path", path)
            except B.StencilError as e:
                res["forms"].append({"path": path, "precision": prec, "t": tt, "unavailable": str(e)})
                continue
            plan.ensure_workspace(x.device)
            sec = _time_runs(lambda: plan.run(x, y, steps), stream, reps=2 if d == 2 else 1)
            info = plan.info()
            res["forms"].append({"path": path, "precision": info["precision_name"], "t": tt,
                                 "gstencils": pts * steps / sec / 1e9,
                                 "model_gstencils": info["predicted_gstencils"], "scenario": info["scenario"]})
            plan.close()
        cu = res["forms"][0].get("gstencils")
        if d == 2 and cu and "gstencils" in res["forms"][1]:
            ratio = res["forms"][1]["gstencils"] / cu
            res["tc_over_cu"] = ratio
            res["measured_change"] = "up" if ratio > 1.05 else ("down" if ratio < 0.95 else "same")
        out.append(res)
        del x, y
        torch.cuda.empty_cache()
    return {"cases": out}


def batched_leg(B, inputs, stream, steps=20, ngrids=512):
    """512 uneven FP32 grids, 4 stencil kinds: one persistent launch replayed
    from a CUDA graph against a per-grid loop of plain stencil_run calls."""
    import numpy as np
    import torch
    descs = inputs.batch_descs()[:ngrids]
    probs = []
    for (shape, r, ny, nx, seed) in descs:
        w = inputs.weights(shape, 2, r, seed)
        probs.append((shape, r, ny, nx, w))
    # fields: one seeded U(0,1) draw per grid (interior), zero halo
    ins, outs = [], []
    for i, (shape, r, ny, nx, w) in enumerate(probs):
        u = inputs.uniform_field((ny, nx), r, descs[i][4], len(w), np.float32)
        ins.append(torch.from_numpy(u).cuda())
        outs.append(torch.empty_like(ins[-1]))
    pts = sum(ny * nx for (_, _, ny, nx, _) in probs)
    batch = B.Batch(probs, "f32", 0)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        # the model's choice per grid, then the autotuned choice per shape class
        sec_model = _time_runs(lambda: batch.run(ins, outs, steps, stream=side, graph=True), side)
        t0 = time.perf_counter()
        tune = batch.autotune(ins, outs, steps, reps=1, stream=side)
        tune_s = time.perf_counter() - t0
        n0 = B.stencil_launch_count()
        batch.run(ins, outs, steps, stream=side, graph=True)  # capture + replay
        side.synchronize()
        n1 = B.stencil_launch_count()
        sec_graph = _time_runs(lambda: batch.run(ins, outs, steps, stream=side, graph=True), side)
        n2 = B.stencil_launch_count()
        sec_batch = _time_runs(lambda: batch.run(ins, outs, steps, stream=side, graph=False), side)
    graph_launches = (n2 - n1) // 4  # per replay (_time_runs: 1 warm + 3 timed)
    chosen = [q for q in tune if q["chosen"]]
    picks = {}
    for q in chosen:
        key = f"{q['path']}:t{q['t']}:{q['tile_y']}x{q['tile_x']}"
        picks[key] = picks.get(key, 0) + q["ngrids"]
    plans = [B.Plan(s, 2, r, w, "f32", (ny, nx), 0) for (s, r, ny, nx, w) in probs]
    for p in plans:
        p.set_option("path", "cuda_core")
        p.ensure_workspace(ins[0].device)

    def loop():
        for p, a, b in zip(plans, ins, outs):
            p.run(a, b, steps)
    n0 = B.stencil_launch_count()
    loop()
    torch.cuda.synchronize()
    loop_launches = B.stencil_launch_count() - n0
    sec_loop = _time_runs(loop, stream, reps=2)
    for p in plans:
        p.close()
    # error of the tuned batched result after `steps` steps against the same
    # grids run as an FP64 batch (FP64 CUDA cores, held within 1e-12 of the
    # oracle by the GPU tests)
    with torch.cuda.stream(side):
        batch.run(ins, outs, steps, stream=side, graph=True)
    side.synchronize()
    batch.close()
    worst = 0.0
    chunk = 128
    for lo in range(0, len(probs), chunk):
        sub = list(range(lo, min(lo + chunk, len(probs))))
        bb = B.Batch([probs[i] for i in sub], "f64", 0)
        i64 = [ins[i].double() for i in sub]
        o64 = [torch.empty_like(a) for a in i64]
        bb.run(i64, o64, steps)
        torch.cuda.synchronize()
        for k, i in enumerate(sub):
            ref = o64[k]
            d = float((outs[i].double() - ref).abs().max() / ref.abs().max().clamp_min(1e-300))
            worst = max(worst, d)
        bb.close()
        del i64, o64
    del ins, outs
    torch.cuda.empty_cache()
    return {"workload": f"{len(probs)} FP32 grids, sides log-uniform in [64, 4096], Star-2D1R/Star-2D2R/Box-2D1R/Box-2D3R, "
                        f"{steps} steps, {pts} interior points",
            "persistent_graph_gstencils": pts * steps / sec_graph / 1e9,
            "persistent_gstencils": pts * steps / sec_batch / 1e9,
            "persistent_graph_model_choice_gstencils": pts * steps / sec_model / 1e9,
            "per_grid_loop_gstencils": pts * steps / sec_loop / 1e9,
            "per_grid_loop_launches": loop_launches, "persistent_graph_kernel_launches": graph_launches,
            "max_rel_linf_vs_fp64": worst,
            "autotune": {"classes": len(chosen), "candidates_measured": sum(1 for q in tune if q["measured_gstencils"] > 0),
                         "seconds": tune_s, "grids_per_choice": picks}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--t", type=int, default=0, help="force the fusion depth (0 = model)")
    ap.add_argument("--path", default="auto")
    ap.add_argument("--precision", default=None)
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-(path, t) sweep")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-precision and batched legs")
    ap.add_argument("--dims", default=None, help="override the interior extents (profiling), e.g. 6144,6144")
    ap.add_argument("--run-steps", type=int, default=None, help="override the steps per run (profiling)")
    ap.add_argument("--leg", default="main", choices=["main", "mixed", "batched", "model", "fusion", "table3"],
                    help="run only the mixed-precision or the batched leg, or the host-only model "
                         "classification, and print its JSON")
    ap.add_argument("--batch-grids", type=int, default=512, help="batched leg: the first N grids (profiling)")
    args = ap.parse_args()

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    cfg = dict(WORKLOADS[args.config])
    if args.dims:
        cfg["dims"] = tuple(int(x) for x in args.dims.split(","))
    if args.run_steps:
        cfg["steps"] = args.run_steps
    if args.impl == "reference":
        return run_reference(args, cfg, args.config, rank)
    if args.leg == "model":  # host arithmetic only: no GPU needed
        from paper_2603_00477_gb300 import binding as B
        from paper_2603_00477_gb300 import build as gbuild
        from paper_2603_00477_gb300 import inputs
        gbuild.build()
        peaks, peaks_src = measured_peaks()
        B.stencil_set_peaks(hbm_bytes_per_s=float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) * 1e9)
        if rank == 0:
            print(json.dumps({"leg": "model", "peaks_source": f"hbm_gbs of {peaks_src} peaks",
                              **model_leg(B, inputs)}))
        return 0

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2603_00477_gb300 import binding as B
    from paper_2603_00477_gb300 import build as gbuild
    from paper_2603_00477_gb300 import inputs

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    gbuild.build()
    B.load()
    peaks, peaks_src = measured_peaks()
    B.stencil_set_peaks(hbm_bytes_per_s=float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS)) * 1e9)
    if args.leg != "main":
        stream = torch.cuda.current_stream()
        if args.leg == "mixed":
            out = mixed_precision_leg(B, inputs, stream)
        elif args.leg == "fusion":
            out = fusion_leg(B, inputs, stream)
        elif args.leg == "table3":
            out = table3_leg(B, inputs, stream)
        else:
            out = batched_leg(B, inputs, stream, ngrids=args.batch_grids)
        if rank == 0:
            print(json.dumps({"leg": args.leg, **out}))
        return 0

    def barrier():
        if world > 1:
            dist.barrier()

    npdt = np.float64 if cfg["dtype"] == "f64" else np.float32
    w, u = inputs.problem(cfg["shape"], cfg["d"], cfg["r"], cfg["dims"], seed=cfg["seed"], dtype=npdt,
                          field=cfg.get("field", "uniform"))
    # CPU baseline (the oracle, no process pool, before any GPU work here)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        oracle.build()
        cpu = cpu_baseline(cfg, w, u)
    plan = B.Plan(cfg["shape"], cfg["d"], cfg["r"], w, cfg["dtype"], cfg["dims"], args.t)
    if args.precision:
        plan.set_option("precision", args.precision)
    if args.path != "auto":
        plan.set_option("path", args.path)
    info = plan.info()
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    plan.ensure_workspace(x.device)
    stream = torch.cuda.current_stream()
    steps = cfg["steps"]
    pts = points_of(cfg)

    for _ in range(args.warmup):
        plan.run(x, y, steps)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    with sampler:
        n0 = B.stencil_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            plan.run(x, y, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        launches = B.stencil_launch_count() - n0
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.summary()
    ms = max_over_ranks(ms, world)
    value = whole_job_rate(world, pts, steps, args.steps, ms / 1e3)

    # roofline of the dominant kernel (the sweep): algorithmic work per launch /
    # average launch duration over the timed region
    t = info["t"]
    nsweeps = steps // t + (1 if steps % t else 0)
    sweep_launches = nsweeps * args.steps
    avg_launch_s = ms / 1e3 / sweep_launches
    K = info["K"]
    D = 8 if cfg["dtype"] == "f64" else 4
    kernel = kernel_name(info, cfg["d"], cfg["dtype"], cfg["shape"], cfg["r"])
    kernel_key = f"{kernel}:{args.config}:{info['path_name']}:t{t}"
    traffic = traffic_record(kernel_key)
    if info["memory_bound"]:
        achieved = pts * 2 * D / avg_launch_s / 1e9  # one read + one write per point and sweep
        peak = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "peak_source": f"hbm_gbs of {peaks_src} peaks"}
    else:
        flops = pts * 2 * K * (steps / nsweeps)  # useful FLOP of one sweep (t steps; remainder averaged)
        achieved = flops / avg_launch_s / 1e12
        peak = ALU_PEAK_TFLOPS[cfg["dtype"]]
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"derived: 152 SMs x 2070 MHz x {'4' if D == 8 else '256'} FLOP/clk/SM "
                               f"({cfg['dtype'].upper()} FMA pipe)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if roof["bound"] == "alu":
        probe = B.stencil_probe_peaks(stream)
        measured = probe["cu_f64_flops" if D == 8 else "cu_f32_flops"] / 1e12
        roof["probe_peak"] = measured
        roof["probe_peak_source"] = ("stencil_probe_peaks: register-only FMA chains on every SM at the maximum "
                                     "clock; for FP64 they reach ~3.2 of the 4 FLOP per SM cycle that this "
                                     "sweep sustains, so the peak above is the derived one")
        roof["probe_frac"] = roof["achieved"] / measured
    roof["traffic"] = traffic
    roof["kernel"] = kernel_key
    roof["avg_launch_ms"] = avg_launch_s * 1e3
    roof["launches_timed"] = sweep_launches

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        # page-locked host buffers from stencil_host_alloc
        h_in = B.host_empty(u.shape, cfg["dtype"])
        h_in.copy_(torch.from_numpy(u))
        h_out = B.host_empty(u.shape, cfg["dtype"])

        def copy_rates():
            # the copy rates of the pinned buffers alone (CUDA events on the
            # stream), each buffer touched once per 4 KiB page first, as
            # stencil_run_host does before its copies
            for hb in (h_in, h_out):
                flat = hb.numpy().reshape(-1)
                float(flat[::4096 // flat.itemsize].sum())
            d_buf = torch.empty(tuple(h_in.shape), dtype=h_in.dtype, device=x.device)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            d_buf.copy_(h_in, non_blocking=True)
            ev[1].record(stream)
            h_out.copy_(d_buf, non_blocking=True)
            ev[2].record(stream)
            torch.cuda.synchronize()
            nb = h_in.numel() * h_in.element_size()
            del d_buf
            return (nb / (max(ev[0].elapsed_time(ev[1]), 1e-6) / 1e3) / 1e9,
                    nb / (max(ev[1].elapsed_time(ev[2]), 1e-6) / 1e3) / 1e9)

        before = copy_rates()
        plan.run_host(h_in, h_out, steps)  # warm (workspace of three grids)
        torch.cuda.synchronize()
        barrier()
        e2e_clocks = ClockSampler(local_rank)
        with e2e_clocks:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                plan.run_host(h_in, h_out, steps)
            el = time.perf_counter() - t0
        el = max_over_ranks(el, world)
        nbytes = h_in.numel() * h_in.element_size()
        e2e = {"value": whole_job_rate(world, pts, steps, args.steps, el), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "api": "stencil_run_host (page-locked host buffers from stencil_host_alloc)",
               "clocks": e2e_clocks.summary()}
        # the copy rates of the same pinned buffers alone, before and after the
        # timed region: they split the end-to-end time into copies and compute
        e2e["h2d_gbs"], e2e["d2h_gbs"] = copy_rates()
        e2e["h2d_gbs_before"], e2e["d2h_gbs_before"] = before
        del h_in, h_out
        plan._ws = None
        torch.cuda.empty_cache()
        plan.ensure_workspace(x.device)

    # FP64 by exact splitting on the tensor cores, against the plain result in y
    split_leg = None
    if not args.no_extras and rank == 0 and cfg["dtype"] == "f64" and cfg["d"] == 2 and \
            info["precision_name"] != "ozaki":
        split_leg = split_fp64_leg(B, cfg, w, x, y, value / world, stream, args.steps)

    # per-(path, t) sweep of the headline workload next to the model's prediction
    sweep = None
    if not args.no_sweep and rank == 0:
        sweep = []
        forms = [("cuda_core", None), ("tensor_core", None)]
        if cfg["dtype"] == "f64":
            forms.append(("tensor_core", "ozaki"))
        for path, prec in forms:
            for tt_ in (1, 2, 3, 4):
                try:
                    p2 = B.Plan(cfg["shape"], cfg["d"], cfg["r"], w, cfg["dtype"], cfg["dims"], tt_)
                    if prec:
                        p2.set_option("precision", prec)
                    p2.set_option("path", path)
                except B.StencilError:
                    continue
                p2._ws = plan._ws
                B.stencil_plan_set_workspace(p2.handle, plan._ws.data_ptr(), plan._ws.numel())
                p2.run(x, y, steps)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                p2.run(x, y, steps)
                b.record(stream)
                torch.cuda.synchronize()
                i2 = p2.info()
                sweep.append({"path": path, "precision": i2["precision_name"], "t": tt_,
                              "gstencils": pts * steps / (a.elapsed_time(b) / 1e3) / 1e9,
                              "model_gstencils": i2["predicted_gstencils"], "alpha": i2["alpha"],
                              "sparsity": i2["sparsity"], "beta": i2["beta"]})
                p2._ws = None
                p2.close()

    extras = {}
    if split_leg is not None:
        extras["mixed_precision_fp64"] = split_leg
    if not args.no_extras and rank == 0 and args.config == DEFAULT and not args.dims:
        del x, y
        plan._ws = None
        torch.cuda.empty_cache()
        extras["mixed_precision"] = mixed_precision_leg(B, inputs, stream)
        extras["batched"] = batched_leg(B, inputs, stream)
        extras["paper_table3_on_gb300"] = table3_leg(B, inputs, stream)
        extras["plain_fp64_gstencils"] = value / world

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": cfg["dtype"],
            "data": "synthetic (seeded splitmix64: weights U(0,1) normalised, field U[0,1))",
            "config": config_json(args.config, cfg, {"parallelism": f"replicas x{world}",
                                                     "path": info["path_name"], "t": t,
                                                     "precision": info["precision_name"],
                                                     "tile": info["tile"]}),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
            "model": {"predicted_gstencils": info["predicted_gstencils"], "scenario": info["scenario"],
                      "intensity": info["intensity"], "ridge": info["ridge"],
                      "memory_bound": bool(info["memory_bound"])},
            "sweep": sweep}
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
