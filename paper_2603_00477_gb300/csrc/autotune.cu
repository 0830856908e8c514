// autotune.cu -- measure the dispatcher's candidates and keep the fastest.
//
// The paper's model (the dispatch rule) ranks (path, precision, t) by their
// roofs; on real hardware the tensor-core path also pays per-instruction and
// operand-bandwidth costs the model does not contain.  The autotuner runs
// every candidate the plan's options allow on the caller's buffers, timed
// with CUDA events on the caller's stream, and makes the fastest the plan's
// choice.  Candidates are visited in the model's order, so the model seeds
// the search and its prediction is reported next to each measurement; 2-D
// CUDA-core candidates are also tried with several tile shapes.
#include <algorithm>
#include <vector>

#include "launch.h"

using namespace gbs;

namespace gbs {
stencil_status dispatch_candidates(Plan *p, std::vector<int> *paths, std::vector<int> *precs, std::vector<int> *ts,
                                   std::vector<double> *model);
}

extern "C" stencil_status stencil_plan_autotune(stencil_plan *plan, const void *in, void *out, int64_t steps, int reps,
                                                stencil_stream_t stream, stencil_tune_result *results, int max_results,
                                                int *n_results)
try {
    if (!plan || !in || !out || steps < 1 || reps < 1)
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_autotune: bad argument");
    Plan &p = plan->p;
    std::vector<int> paths, precs, ts;
    std::vector<double> model;
    stencil_status s = dispatch_candidates(&p, &paths, &precs, &ts, &model);
    if (s != STENCIL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(STENCIL_ERR_CUDA, "stencil_plan_autotune: cudaEventCreate");
    const Plan saved = p;
    double best = -1;
    size_t best_i = 0;
    int best_tile[2] = {0, 0};
    int n = 0;
    // CUDA-core candidates of a 2-D plan are also tried with other tile shapes
    // (the default first); the tile changes the redundant halo work of the
    // overlapped temporal tiles and the occupancy
    static const int kTiles2d[][2] = {{0, 0}, {32, 256}, {64, 128}, {64, 64}, {32, 128}, {128, 64}};
    struct Trial {
        size_t i;
        int ty, tx;
    };
    std::vector<Trial> trials;
    size_t def_i = (size_t)-1;
    int def_tile[2] = {0, 0};
    for (size_t i = 0; i < paths.size(); i++) {
        if (paths[i] == STENCIL_PATH_CUDA_CORE && saved.pat.d == 2 && !saved.req_tile[1]) {
            for (auto &tl : kTiles2d) trials.push_back({i, tl[0], tl[1]});
        } else {
            trials.push_back({i, 0, 0});
        }
    }
    for (const Trial &tr : trials) {
        const size_t i = tr.i;
        Plan trial = saved;
        trial.req_path = paths[i];
        trial.req_precision = precs[i];
        trial.req_t = ts[i];
        trial.req_tile[0] = trial.req_tile[1] = trial.req_tile[2] = 0;
        if (tr.ty) {
            trial.req_tile[0] = 1;
            trial.req_tile[1] = tr.ty;
            trial.req_tile[2] = tr.tx;
        }
        if (dispatch(&trial) != STENCIL_OK) continue;
        if (!tr.ty) {  // the candidate's default tile, tried first
            def_i = i;
            def_tile[0] = trial.tile[1];
            def_tile[1] = trial.tile[2];
        } else if (def_i == i && trial.tile[1] == def_tile[0] && trial.tile[2] == def_tile[1]) {
            continue;  // the default tile again
        }
        p = trial;
        s = stencil_run(plan, in, out, steps, stream);  // warm-up
        if (s == STENCIL_ERR_UNSUPPORTED && tr.ty) {  // this tile does not fit shared memory
            s = STENCIL_OK;
            continue;
        }
        if (s != STENCIL_OK) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == STENCIL_OK; r++) s = stencil_run(plan, in, out, steps, stream);
        cudaEventRecord(e1, st);
        if (s != STENCIL_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "stencil_plan_autotune: timing");
            break;
        }
        const double gst = (double)p.n_interior * steps * reps / (ms * 1e-3) / 1e9;
        if (results && n < max_results) {
            results[n].path = paths[i];
            results[n].precision = precs[i];
            results[n].t = ts[i];
            results[n].model_gstencils = trial.info.predicted_gstencils;
            results[n].measured_gstencils = gst;
            results[n].tile_y = trial.tile[1];
            results[n].tile_x = trial.tile[2];
        }
        n++;
        if (gst > best) {
            best = gst;
            best_i = i;
            best_tile[0] = tr.ty;
            best_tile[1] = tr.tx;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results) *n_results = n;
    if (s != STENCIL_OK || best < 0) {
        p = saved;
        return s != STENCIL_OK ? s : fail(STENCIL_ERR_UNSUPPORTED, "stencil_plan_autotune: no candidate ran");
    }
    Plan chosen = saved;
    chosen.req_path = paths[best_i];
    chosen.req_precision = precs[best_i];
    chosen.req_t = ts[best_i];
    chosen.req_tile[0] = chosen.req_tile[1] = chosen.req_tile[2] = 0;
    if (best_tile[0]) {
        chosen.req_tile[0] = 1;
        chosen.req_tile[1] = best_tile[0];
        chosen.req_tile[2] = best_tile[1];
    }
    s = dispatch(&chosen);
    if (s != STENCIL_OK) {
        p = saved;
        return s;
    }
    p = chosen;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_autotune");
}
