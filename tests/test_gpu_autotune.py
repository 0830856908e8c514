"""GPU test of the model-seeded autotuner: it measures every candidate the
plan's options allow, keeps the fastest, and the plan then runs that choice
bit for bit like a plan created with the same (path, precision, t)."""
import numpy as np
import pytest

from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


@pytest.mark.parametrize("shape,r,dtype,prec", [("box", 2, "f32", "any"), ("box", 3, "f64", "native"),
                                                ("star", 2, "f32", "native")])
def test_autotune_picks_fastest_and_runs_it(torch, shape, r, dtype, prec):
    dims = (700, 900)
    npdt = np.float64 if dtype == "f64" else np.float32
    w, u = inputs.problem(shape, 2, r, dims, seed=77, dtype=npdt)
    plan = B.Plan(shape, 2, r, w, dtype, dims)
    if dtype == "f32":
        plan.set_option("precision", prec)
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    res = plan.autotune(x, y, steps=4, reps=1)
    assert len(res) >= 2
    assert all(q["measured_gstencils"] > 0 and q["model_gstencils"] > 0 for q in res)
    # candidates are visited in the model's order (each first with its default tile)
    firsts, seen = [], set()
    for q in res:
        key = (q["path"], q["precision"], q["t"])
        if key not in seen:
            seen.add(key)
            firsts.append(q["model_gstencils"])
    assert firsts == sorted(firsts, reverse=True)
    best = max(res, key=lambda q: q["measured_gstencils"])
    info = plan.info()
    assert (info["path_name"], info["precision_name"], info["t"]) == (best["path"], best["precision"], best["t"])
    assert tuple(info["tile"][1:]) == tuple(best["tile"])
    if best["path"] == "cuda_core":
        assert len({q["tile"] for q in res if q["path"] == "cuda_core" and q["t"] == best["t"]}) >= 2
    if prec == "native":
        assert best["precision"] == "native"
    plan.run(x, y, 5)
    got = y.cpu().numpy()

    ref_plan = B.Plan(shape, 2, r, w, dtype, dims, best["t"])
    if dtype == "f32":
        ref_plan.set_option("precision", best["precision"])
    ref_plan.set_option("path", best["path"])
    if best["path"] == "cuda_core":
        ref_plan.set_option("tile", f"{best['tile'][0]}x{best['tile'][1]}")
    z = torch.empty_like(x)
    ref_plan.run(x, z, 5)
    B.stencil_device_status()
    np.testing.assert_array_equal(got, z.cpu().numpy())
    plan.close()
    ref_plan.close()


def test_autotune_rejects_bad_arguments(torch):
    w = inputs.weights("box", 2, 1, seed=1)
    plan = B.Plan("box", 2, 1, w, "f64", (64, 64))
    x = torch.zeros(plan.stored_shape, dtype=torch.float64, device="cuda")
    with pytest.raises(B.StencilError) as e:
        B.stencil_plan_autotune(plan.handle, x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status == B.STENCIL_ERR_INVALID_ARG
    plan.close()
