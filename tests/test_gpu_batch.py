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
