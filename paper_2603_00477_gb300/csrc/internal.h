// internal.h -- host-side structures shared by the translation units of
// libgbstencil (plan, model, dispatch, launchers).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "gbstencil.h"

namespace gbs {

constexpr int kMaxT = 16;

// Pattern description.  Offsets are listed in the order the weights follow:
// lexicographic, first axis outermost, each coordinate ascending from -r.
struct Pattern {
    int shape = 0;  // STENCIL_BOX / STENCIL_STAR
    int d = 0;
    int r = 0;
    int K = 0;
    std::vector<int> offs;  // K * d
};

bool make_pattern(int shape, int d, int r, Pattern *p);
int pattern_points(int shape, int d, int r);

// Dense composite kernel w^(t) (box of radius t*r, (2tr+1)^d values, same
// lexicographic order), FP64.  t = 0 gives the identity.
std::vector<double> compose_dense(const Pattern &p, const std::vector<double> &w, int t);

// ---- performance model (paper Sec. 3-4) ----
struct ModelOut {
    int K = 0, K_fused = 0;
    double alpha = 1, C_cu = 0, C_tc = 0, M = 0, I_cu = 0, I_tc = 0;
    double ridge_cu = 0, ridge_tc = 0, P_cu_actual = 0, P_tc_actual = 0, speedup = 0;
    int scenario = 0, sweet_spot = 0;
    double gst_cu = 0, gst_tc = 0;
};
int fused_points(int shape, int d, int r, int t);
ModelOut model_eval(int shape, int d, int r, int t, int D, double S, double beta, double P_cu,
                    double P_tc, double B);

stencil_peaks peaks();  // a copy of the process-wide table (thread safe)

// ---- tensor-core tile geometry (host view of what the TC kernels issue) ----
struct TcGeometry {
    bool available = false;
    int n_tile = 0;      // MMA N (output columns per accumulator)
    int k_inst = 0;      // MMA K per instruction
    int kext = 0;        // K extent per row offset (window, padded)
    double sparsity = 0; // useful / issued MACs of the B tiles
};
TcGeometry tc_geometry(int shape, int d, int r, int t, stencil_dtype dtype, int precision, int path);

// ---- FP64 by exact splitting (k_split.cu) ----
// Digit slices S (6 or 7) of the plan's composite kernel at depth t for
// which every product level sums exactly in FP32; 0 if none (or 2-D FP64
// with t*r <= 8 does not hold).  Host only.
int split_slices(const struct Plan &p, int t);
// Output column blocks of 16 per tile that fit in shared memory (0: none).
int split_nacc(int R, int S);

// ---- plan ----
struct Plan {
    Pattern pat;
    stencil_dtype dtype = STENCIL_F64;
    int64_t dims[3] = {1, 1, 1};  // interior, slowest first (d used)
    int64_t ext[3] = {1, 1, 1};   // stored extents
    int64_t n_interior = 0, n_stored = 0;
    std::vector<double> w;

    // user requests
    int req_path = STENCIL_PATH_AUTO;
    int req_precision = STENCIL_PREC_NATIVE;
    int req_t = 0;
    int req_tile[3] = {0, 0, 0};
    int debug_unmet_wait = 0;  // test hook for the tensor-core kernels' bounded wait

    // decision
    int path = STENCIL_PATH_CUDA_CORE;
    int precision = STENCIL_PREC_NATIVE;
    int t = 1;
    int tile[3] = {1, 1, 1};
    stencil_info info{};

    // device workspace (caller owned)
    void *ws = nullptr;
    size_t ws_bytes = 0;

    size_t elem_bytes() const { return dtype == STENCIL_F64 ? 8 : 4; }
    size_t grid_bytes() const { return (size_t)n_stored * elem_bytes(); }
};

stencil_status dispatch(Plan *p);  // fills path/precision/t/tile/info

// kernel-family availability (host knowledge of what the .cu files build)
bool cu_supported(int shape, int d, int r);
void cu_default_tile(const Plan &p, int t, int tile[3]);
bool tc_supported(const Plan &p, int precision, int path);

// ---- errors ----
stencil_status fail(stencil_status s, const std::string &msg);
// Status for a C++ exception caught at ABI entry point `entry` (call from
// inside the handler): std::bad_alloc / std::length_error -> OOM, anything
// else -> INTERNAL; records the message without allocating if it cannot.
stencil_status abi_exception(const char *entry) noexcept;
void note_launch(uint64_t n = 1);

}  // namespace gbs

struct stencil_plan {
    gbs::Plan p;
};
