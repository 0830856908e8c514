"""The host-only model leg of bench.py (`--leg model`): the paper's problem
classification (CUDA-core intensity of Eq. 8 against the ridge point, t = 1..8)
and its six representative cases, evaluated by the library with GB300's peak
table and this engine's own MMA tiles.  Checked against the oracle's copy of
the model, against what GB300's unit rates fix, and against the intensity the
paper prints for the sparse cases (Sec. 5.3, reproduced by the engine's
2:4 layout because its S equals the one the paper uses there).  No kernel
runs."""
import importlib
import json
import math
import os

import pytest

from oracle import model
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import build as gbuild
from paper_2603_00477_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
HBM = 6.8e12


@pytest.fixture(scope="module")
def leg():
    gbuild.build()
    B.load()
    old = B.stencil_get_peaks()
    bench = importlib.import_module("bench")
    try:
        B.stencil_set_peaks(hbm_bytes_per_s=HBM)
        out = bench.model_leg(B, inputs)
        json.dumps(out)  # the leg prints this as one JSON line
        yield out
    finally:
        B.stencil_set_peaks(**old)


def _parse(name):
    shape, rest = name.split("-")
    return shape.lower(), int(rest[0]), int(rest[2:-1])


def test_classification_matches_oracle_model(leg):
    P = {"f32": leg["peaks"]["cu_f32_flops"], "f64": leg["peaks"]["cu_f64_flops"]}
    for dtype, rows in leg["classification"].items():
        D = 4 if dtype == "f32" else 8
        for row in rows:
            shape, d, r = _parse(row["stencil"])
            for t in range(1, leg["tmax"] + 1):
                I = model.I_cu(shape, d, r, t, D)
                assert row["I"][t - 1] == pytest.approx(I, rel=1e-14)
                want = "compute" if model.bound(I, P[dtype], HBM) == "CB" else "memory"
                assert row["bound"][t - 1] == want, (dtype, row["stencil"], t)
            first = row["compute_bound_from_t"]
            assert first is None or row["bound"][first - 1] == "compute"
            assert all(b == "memory" for b in row["bound"][:(first or leg["tmax"] + 1) - 1])


def test_fp64_is_compute_bound_everywhere(leg):
    """GB300's FP64 FMA rate (about 1.26 TFLOP/s) puts the ridge near
    0.19 FLOP/B, below the intensity of the smallest stencil (Star-2D1R,
    10/16): no FP64 configuration is memory bound, so fusion never pays."""
    for row in leg["classification"]["f64"]:
        assert row["compute_bound_from_t"] == 1
        assert row["ridge"] < 0.2


def test_fp32_transition_ordering(leg):
    """Sec. 4.2's reading of the classification: a higher dimension or a
    larger radius needs fewer fused steps to become compute bound, and
    Box-3D2R is compute bound without fusion."""
    rows = {r["stencil"]: r["compute_bound_from_t"] or math.inf for r in leg["classification"]["f32"]}
    assert rows["Box-3D2R"] == 1
    for shape in ("Box", "Star"):
        radii = [rows[f"{shape}-2D{r}R"] for r in (1, 2, 3, 7)]
        assert radii == sorted(radii, reverse=True)
        for r in (1, 2):
            assert rows[f"{shape}-3D{r}R"] <= rows[f"{shape}-2D{r}R"]
    # I = K t / 4 on FP32 storage: the first compute-bound t is ceil(4 ridge / K)
    ridge = leg["peaks"]["cu_f32_flops"] / HBM
    for name, first in rows.items():
        shape, d, r = _parse(name)
        t = math.ceil(4 * ridge / model.K_points(shape, d, r))
        assert first == (t if t <= leg["tmax"] else math.inf), name


def test_paper_cases(leg):
    with open(os.path.join(GOLDEN, "paper_table3.json")) as f:
        printed = {c["case"]: c for c in json.load(f)["cases"]}
    assert len(leg["cases"]) == 6
    for i, case in enumerate(leg["cases"], 1):
        p = printed[i]
        shape, d, r = _parse(case["stencil"])
        assert (shape, d, r, case["t"]) == (p["shape"], p["d"], p["r"], p["t"])
        assert case["dtype"] == ("f64" if p["D"] == 8 else "f32")
        cu = case["cuda_core"]
        assert cu["path_name"] == "cuda_core" and cu["t"] == p["t"]
        if i != 4:  # case 4's printed CU intensity disagrees with Table 2 (56.25)
            assert cu["intensity"] == pytest.approx(p["I_cu"], abs=0.006)
        tc = case["tensor_core"]
        if d == 3:
            assert tc is None and case["tensor_core_unavailable"]  # no 3-D tensor-core tiles
            continue
        D = p["D"]
        if D == 8:
            # FP64 MMA runs at the FP64 FMA rate on GB300: always scenario 4,
            # and the redundancy alpha/S makes it lose
            assert tc["path_name"] == "tensor_core" and case["scenario"] == 4
            assert tc["predicted_gstencils"] < cu["roof_gstencils"]
        else:
            # the 2:4 layout's S for R = 7 is the 15/32 the paper uses for
            # SPIDER, so the tensor-core intensity is the printed 120.00
            assert tc["path_name"] == "sparse_tensor_core"
            assert tc["sparsity"] == pytest.approx(15 / 32)
            assert tc["intensity"] == pytest.approx(p["I_tc"], abs=0.006)
            assert case["scenario"] == p["scenario"] == 3
            assert tc["predicted_gstencils"] > cu["roof_gstencils"]
        S = tc["sparsity"]
        P_cu = leg["peaks"]["cu_f64_flops" if D == 8 else "cu_f32_flops"]
        P_tc = leg["peaks"]["tc_f64_flops" if D == 8 else "sptc_tf32_flops"]
        assert case["scenario"] == model.scenario(shape, d, r, p["t"], D, S, P_cu, P_tc, HBM)
        assert tc["intensity"] == pytest.approx(model.I_tc(shape, d, r, p["t"], D, S), rel=1e-12)


def test_cli_prints_one_json_line():
    """`bench.py --leg model` needs no GPU and prints one JSON line."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--leg", "model"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert res.returncode == 0, res.stderr
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["leg"] == "model" and len(out["cases"]) == 6
    assert set(out["classification"]) == {"f32", "f64"}


def test_kernel_names():
    """The bench names the sweep kernel a plan launches by the launchers' rules:
    3-D t = 1 FP32 star r <= 3 / box r = 1 on the rotating kernel, the FP16 /
    BF16 forms on the wide kernel, 3-D FP16 on its z-marching form."""
    bench = importlib.import_module("bench")
    kn = bench.kernel_name
    assert kn({"path": 1, "t": 1, "precision_name": "native"}, 2, "f64") == "cu2d_sweep"
    assert kn({"path": 1, "t": 1, "precision_name": "native"}, 3, "f32", "star", 2) == "cu3d_rot"
    assert kn({"path": 1, "t": 1, "precision_name": "native"}, 3, "f32", "box", 1) == "cu3d_rot"
    assert kn({"path": 1, "t": 1, "precision_name": "native"}, 3, "f32", "box", 2) == "cu3d_stream"
    assert kn({"path": 1, "t": 1, "precision_name": "native"}, 3, "f64", "star", 2) == "cu3d_stream"
    assert kn({"path": 1, "t": 2, "precision_name": "native"}, 3, "f64") == "cu3d_sweep"
    assert kn({"path": 2, "t": 2, "precision_name": "native"}, 2, "f64") == "dmma2d_sweep"
    assert kn({"path": 2, "t": 1, "precision_name": "ozaki"}, 2, "f64") == "tc2d_split"
    assert kn({"path": 2, "t": 4, "precision_name": "tf32"}, 2, "f32") == "tc2d_ws"
    assert kn({"path": 2, "t": 2, "precision_name": "bf16x3", "tile": [1, 128, 128]}, 2, "f32") == "tc2d_wide"
    assert kn({"path": 2, "t": 4, "precision_name": "f16", "tile": [1, 256, 128]}, 2, "f32") == "tc2d_wide"
    assert kn({"path": 2, "t": 6, "precision_name": "f16x3", "tile": [1, 128, 128]}, 2, "f32") == "tc2d_wide"
    assert kn({"path": 3, "t": 3, "precision_name": "tf32"}, 2, "f32") == "sptc2d_sweep"
    assert kn({"path": 2, "t": 1, "precision_name": "f16", "tile": [1, 128, 128]}, 3, "f32", "box", 1) == "tc3d_wide"
