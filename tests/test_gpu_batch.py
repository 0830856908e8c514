"""GPU parity of the batched form (one persistent launch over many uneven
grids with mixed stencils) against the FP64 oracle and, bit for bit, against
running each grid alone through stencil_run with the same fusion depth."""
import numpy as np
import pytest

import oracle
from paper_2603_00477_gb300 import binding as B
from paper_2603_00477_gb300 import inputs

pytestmark = pytest.mark.gpu

GRIDS = [("star", 1, 1, 1), ("box", 3, 200, 37), ("star", 2, 65, 129), ("box", 1, 300, 250), ("box", 2, 5, 400),
         ("star", 3, 128, 64), ("box", 1, 63, 65), ("star", 1, 777, 33), ("box", 3, 2, 2), ("star", 2, 140, 140)]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_2603_00477_gb300 import build
    build.build()
    B.load()
    return _t


def _problems(dtype, seed0=500):
    npdt = np.float64 if dtype == "f64" else np.float32
    out = []
    for i, (shape, r, ny, nx) in enumerate(GRIDS):
        w, u = inputs.problem(shape, 2, r, (ny, nx), seed=seed0 + i, dtype=npdt)
        out.append((shape, r, ny, nx, w, u))
    return out


@pytest.mark.parametrize("dtype,t,steps", [("f32", 0, 7), ("f64", 2, 5), ("f32", 3, 9), ("f32", 1, 1)])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_matches_oracle_and_single_runs(torch, dtype, t, steps, graph):
    probs = _problems(dtype)
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], dtype, t)
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.full_like(x, float("nan")) for x in ins]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(ins, outs, steps, stream=stream, graph=graph)
        if graph:  # the replay must give the same result
            for y in outs:
                y.fill_(float("nan"))
            batch.run(ins, outs, steps, stream=stream, graph=graph)
    B.stencil_batch_status(batch.handle, stream)
    tol = 1e-12 if dtype == "f64" else 1e-5
    for i, (shape, r, ny, nx, w, u) in enumerate(probs):
        got = outs[i].cpu().numpy()
        ref = oracle.run(shape, 2, r, w, (ny, nx), u.astype(np.float64), steps)
        assert oracle.rel_linf(got, ref) <= tol, (i, shape, r, ny, nx)
        assert not np.isnan(got).any()
        # the same grid alone, same t, through stencil_run: identical bits
        info = batch.info(i)
        plan = B.Plan(shape, 2, r, w, dtype, (ny, nx), info["t"])
        plan.set_option("path", "cuda_core")
        y1 = torch.empty_like(ins[i])
        plan.run(ins[i], y1, steps)
        torch.cuda.synchronize()
        assert np.array_equal(y1.cpu().numpy(), got), i
        plan.close()
    batch.close()


def test_batch_steps_zero_and_rejects(torch):
    probs = _problems("f32")
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 0)
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.empty_like(x) for x in ins]
    batch.run(ins, outs, 0)
    torch.cuda.synchronize()
    for x, y in zip(ins, outs):
        assert torch.equal(x, y)
    with pytest.raises(B.StencilError) as e:
        B.stencil_batch_run(batch.handle, [x.data_ptr() for x in ins], [x.data_ptr() for x in ins], 3)
    assert e.value.status == B.STENCIL_ERR_INVALID_ARG
    batch.close()


def test_batch_uneven_config_sample(torch):
    """The uneven 512-grid configuration (sides log-uniform in [64, 4096], four
    stencil kinds, FP32): the first 24 grids, 20 steps, against the oracle."""
    descs = inputs.batch_descs()[:24]
    probs = []
    for (shape, r, ny, nx, seed) in descs:
        w, u = inputs.problem(shape, 2, r, (ny, nx), seed=seed, dtype=np.float32)
        probs.append((shape, r, ny, nx, w, u))
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 0)
    ins = [torch.from_numpy(u).cuda() for (*_, u) in probs]
    outs = [torch.empty_like(x) for x in ins]
    batch.run(ins, outs, 20)
    B.stencil_batch_status(batch.handle)
    for i, (shape, r, ny, nx, w, u) in enumerate(probs):
        lo = (ny // 2, nx // 2)
        hi = (min(ny, lo[0] + 3), min(nx, lo[1] + 3))
        ref = oracle.run_region(shape, 2, r, w, (ny, nx), u.astype(np.float64), 20, lo, hi)
        got = outs[i][lo[0] + r:hi[0] + r, lo[1] + r:hi[1] + r].cpu().numpy()
        assert oracle.rel_linf(got, ref) <= 1e-5, i
        ref0 = oracle.run_region(shape, 2, r, w, (ny, nx), u.astype(np.float64), 20, (0, 0), (2, 2))
        got0 = outs[i][r:r + 2, r:r + 2].cpu().numpy()
        assert np.max(np.abs(got0 - ref0)) <= 1e-5 * max(1e-30, float(np.max(np.abs(ref)))), i
    batch.close()


def _mixed(n, seed, lo, hi, big=()):
    """n grids of the four batched stencil kinds, sides log-uniform in [lo, hi],
    plus the `big` (ny, nx) grids (Box-2D2R)."""
    rng = np.random.default_rng(seed)
    kinds = [("star", 1), ("star", 2), ("box", 1), ("box", 3)]
    out = []
    for i in range(n):
        shape, r = kinds[i % 4]
        ny, nx = (int(np.exp(rng.uniform(np.log(lo), np.log(hi)))) for _ in range(2))
        w, u = inputs.problem(shape, 2, r, (ny, nx), seed=900 + i, dtype=np.float32)
        out.append((shape, r, ny, nx, w, u))
    for j, (ny, nx) in enumerate(big):
        w, u = inputs.problem("box", 2, 2, (ny, nx), seed=950 + j, dtype=np.float32)
        out.append(("box", 2, ny, nx, w, u))
    return out


def _size_class(ny, nx):
    return min(6, max(0, int(np.floor(np.log2(ny * nx) / 2)) - 6))


def _bound(info, shape, r, w, ny, nx, steps):
    """Tolerance of a grid's result: FP32 CUDA cores 1e-5; a tensor-core form
    its derived bound."""
    from tc_bounds import sp_bound, tc_bound
    if info["path"] == B.PATH_CUDA_CORE:
        return 1e-5
    plan = B.Plan(shape, 2, r, w, "f32", (ny, nx), info["t"])
    form = B.PREC_NAMES[info["precision"]]
    if info["path"] == B.PATH_SPARSE_TENSOR_CORE:
        b = sp_bound(plan.handle, shape, r, steps, info["t"])
    else:
        plan.set_option("precision", form)
        b = tc_bound(form, steps, info["t"], plan.handle, shape, r)
    plan.close()
    return b


def _check_all(torch, batch, probs, outs, steps):
    for i, (shape, r, ny, nx, w, u) in enumerate(probs):
        got = outs[i].cpu().numpy()
        ref = oracle.run(shape, 2, r, w, (ny, nx), u.astype(np.float64), steps)
        tol = _bound(batch.info(i), shape, r, w, ny, nx, steps)
        assert oracle.rel_linf(got, ref) <= tol, (i, shape, r, ny, nx, batch.info(i)["path"])
        assert not np.isnan(got).any()


def test_batch_autotune_per_shape_class(torch):
    """The autotuner measures each shape class's candidates (model order, plus
    the current choice), gives every grid of the class the fastest, and the
    tuned batch still matches the oracle."""
    probs = _mixed(16, 77, 64, 700)
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 0)
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.empty_like(x) for x in ins]
    steps = 6
    res = batch.autotune(ins, outs, steps, reps=1)
    classes = {}
    for q in res:
        classes.setdefault(q["cls"], []).append(q)
    keys = {(s, r, _size_class(ny, nx)) for (s, r, ny, nx, _, _) in probs}
    assert len(classes) == len(keys)
    for rows in classes.values():
        ran = [q for q in rows if q["measured_gstencils"] > 0]
        chosen = [q for q in rows if q["chosen"]]
        assert len(chosen) == 1 and ran
        assert chosen[0]["measured_gstencils"] == max(q["measured_gstencils"] for q in ran)
        for path in {q["path"] for q in rows}:  # each path's rows in the model's order (then the current choice)
            model = [q["model_gstencils"] for q in rows if q["path"] == path]
            assert model[:-1] == sorted(model[:-1], reverse=True)
        assert all(q["path"] == "cuda_core" for q in rows)  # native precision: CUDA cores only
        c = chosen[0]
        members = [i for i, (s, r, ny, nx, _, _) in enumerate(probs)
                   if (s, r, _size_class(ny, nx)) == (c["shape"], c["r"], c["size_class"])]
        assert len(members) == c["ngrids"]
        for i in members:
            info = batch.info(i)
            assert (info["t"], info["tile"][1], info["tile"][2]) == (c["t"], c["tile_y"], c["tile_x"])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for y in outs:
            y.fill_(float("nan"))
        batch.run(ins, outs, steps, stream=stream, graph=True)
    B.stencil_batch_status(batch.handle, stream)
    _check_all(torch, batch, probs, outs, steps)
    batch.close()


def test_batch_tensor_core_grids_run_inside_the_graph(torch):
    """Grids put on the tensor-core path run as their own sweeps after the
    persistent kernel, captured in the same graph; every kernel node counts."""
    probs = _mixed(4, 31, 100, 400)
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 0)
    batch.set_option("precision", "tf32x3")
    batch.set_option("path", "tensor_core")
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.full_like(x, float("nan")) for x in ins]
    steps = 5
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(ins, outs, steps, stream=stream, graph=True)  # capture + first replay
        stream.synchronize()
        for y in outs:
            y.fill_(float("nan"))
        n0 = B.stencil_launch_count()
        batch.run(ins, outs, steps, stream=stream, graph=True)  # replay only
        n1 = B.stencil_launch_count()
    B.stencil_batch_status(batch.handle, stream)
    assert n1 - n0 > len(probs)  # at least a halo copy and a sweep per grid
    for i in range(len(probs)):
        assert batch.info(i)["path"] == B.PATH_TENSOR_CORE
    _check_all(torch, batch, probs, outs, steps)
    batch.close()


def test_batch_autotune_may_choose_tensor_cores(torch):
    """With precision "any", large grids' classes also measure the dense and
    sparse tensor-core forms; whatever wins, the result meets its bound."""
    probs = _mixed(6, 5, 64, 300, big=[(600, 640), (700, 560)])
    batch = B.Batch([(s, r, ny, nx, w) for (s, r, ny, nx, w, _) in probs], "f32", 0)
    batch.set_option("precision", "any")
    ins = [torch.from_numpy(u.copy()).cuda() for (*_, u) in probs]
    outs = [torch.empty_like(x) for x in ins]
    steps = 8
    res = batch.autotune(ins, outs, steps, reps=1)
    big = [q for q in res if q["shape"] == "box" and q["r"] == 2 and q["size_class"] >= 3]
    assert {q["path"] for q in big} >= {"cuda_core", "tensor_core", "sparse_tensor_core"}
    small = [q for q in res if q["size_class"] < 3]
    assert all(q["path"] == "cuda_core" for q in small)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(ins, outs, steps, stream=stream, graph=True)
    B.stencil_batch_status(batch.handle, stream)
    _check_all(torch, batch, probs, outs, steps)
    batch.close()
