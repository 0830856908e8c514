// plan.cpp -- plan creation, options, dispatch and diagnostics (host only).
//
// Dispatch is the paper's model used as a decision rule: for every
// available (path, precision, t) the attainable point-update rate is
// min(P S / (2K alpha beta), t B / (2D)) (Eq. 8 for CUDA cores, Eq. 12 for
// tensor cores, Eq. 20 with the sparse peak), the CUDA-core compute term
// being divided by the redundant work of overlapped temporal tiles (the
// halo overlap the paper leaves out of its model), and the tensor-core term
// capped by an instruction-level roof (the MMA-shape efficiency below).  The fastest candidate
// wins; candidates within 2 % of it are ordered CUDA cores first (no
// redundancy), then smaller t, then fewer products.
#include <algorithm>
#include <atomic>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <new>
#include <stdexcept>
#include <string>

#include <cuda_runtime.h>

#include "internal.h"
#include "tc_layout.h"

namespace gbs {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

stencil_status fail(stencil_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

stencil_status abi_exception(const char *entry) noexcept
{
    stencil_status s = STENCIL_ERR_INTERNAL;
    const char *what = "unknown exception";
    try {
        throw;
    } catch (const std::bad_alloc &) {
        s = STENCIL_ERR_OOM;
        what = "host allocation failed";
    } catch (const std::length_error &) {
        s = STENCIL_ERR_OOM;
        what = "host allocation too large";
    } catch (const std::exception &e) {
        what = e.what();
    } catch (...) {
    }
    try {
        g_last_error = std::string(entry) + ": " + what;
    } catch (...) {
        g_last_error.clear();
    }
    return s;
}

void note_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Radii the CUDA-core kernels are instantiated for (k_cuda_core*.cu).
bool cu_supported(int shape, int d, int r)
{
    if (d == 2) return r >= 1 && r <= 7;
    if (d == 3) return shape == STENCIL_BOX ? (r >= 1 && r <= 2) : (r >= 1 && r <= 4);
    return false;
}

// Largest t the dispatcher considers on its own (an explicit t may be larger).
// 3-D: one step per sweep.  The streaming t = 1 kernel reads each plane once
// per tile (only the y/x halo is re-read); fused 3-D tiles re-read
// (T + 2tR)^3 / T^3 of the grid per sweep, which the model's one-read-one-
// write memory term leaves out (measured on GB300: 2-20x slower than t = 1).
static int max_fused_t(const Plan &p, int path)
{
    if (path == STENCIL_PATH_CUDA_CORE) return p.pat.d == 2 ? 4 : 1;
    return 4;
}

// SMs of the current device (152 when no device answers: host-only use).
static int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();  // clear the error of a host without a device
        return 152;
    }
    return sms;
}

void cu_default_tile(const Plan &p, int t, int tile[3])
{
    const int R = p.pat.r;
    if (p.pat.d == 2) {
        tile[0] = 1;
        tile[1] = 64;
        tile[2] = p.dtype == STENCIL_F64 ? 64 : 128;
        if (p.dtype == STENCIL_F32 && t == 1 && R <= 2) {
            // one FP32 sub-step of a small stencil: a wider, flatter tile
            // (measured 2-4 % faster on GB300 than 64 x 128)
            tile[1] = 32;
            tile[2] = 256;
        }
        // two staging buffers (+ a work buffer for t > 1) under ~112 KB, so
        // that two CTAs share an SM
        for (;;) {
            size_t h = tile[1] + 2 * t * R, w = tile[2] + 2 * t * R;
            size_t bytes = h * w * p.elem_bytes() * (t > 1 ? 3 : 2);
            if (bytes <= 112 * 1024 || (tile[2] <= 16 && tile[1] <= 16)) break;
            if (tile[2] >= tile[1]) tile[2] /= 2; else tile[1] /= 2;
        }
        // small grids: at least two tiles per SM (down to 16 x 32 tiles), so
        // that a sweep of a few hundred thousand points is not a few CTAs' work
        const int64_t want = 2 * (int64_t)device_sms();
        auto ntiles = [&] {
            return ((p.dims[1] + tile[1] - 1) / tile[1]) * ((p.dims[2] + tile[2] - 1) / tile[2]);
        };
        while (ntiles() < want) {
            if (tile[2] >= tile[1] && tile[2] > 32) tile[2] /= 2;
            else if (tile[1] > 16) tile[1] /= 2;
            else break;
        }
    } else if (t == 1) {
        // the streaming kernels: runs of planes (64 nominal; the rotating
        // FP32 kernel sizes them to the resident CTAs) of a (16 RPT) x 64 tile
        tile[0] = 64;
        tile[1] = p.dtype == STENCIL_F64 ? 16 : 32;
        if (p.dtype == STENCIL_F32 && p.pat.shape == STENCIL_STAR && R == 3) tile[1] = 16;
        tile[2] = 64;
    } else {
        tile[0] = 8;
        tile[1] = 8;
        tile[2] = 32;
        for (;;) {
            size_t z = tile[0] + 2 * t * R, h = tile[1] + 2 * t * R, w = tile[2] + 2 * t * R;
            size_t bytes = z * h * w * p.elem_bytes() * (t > 1 ? 3 : 2);
            if (bytes <= 112 * 1024 || (tile[0] <= 2 && tile[1] <= 4 && tile[2] <= 8)) break;
            if (tile[0] > 2) tile[0] /= 2;
            else if (tile[1] > 4) tile[1] /= 2;
            else tile[2] /= 2;
        }
    }
}

// Issued-work factor of overlapped temporal tiles: sub-step s computes the
// tile grown by (t - s) r on every side.
static double cu_overlap_factor(const Plan &p, int t, const int tile[3])
{
    const int d = p.pat.d, r = p.pat.r;
    double issued = 0, useful = (double)t;
    for (int s = 1; s <= t; s++) {
        double v = 1;
        for (int i = 3 - d; i < 3; i++) v *= (double)(tile[i] + 2 * (t - s) * r) / tile[i];
        issued += v;
    }
    return issued / useful;
}

// Lines (rows in 2-D, (plane,row) pairs in 3-D) of the composite kernel and
// the half-width of each: box lines are all R wide; a star line at plane c,
// row a holds |b| <= r (t - ceil|c|/r - ceil|a|/r).
static void composite_lines(int shape, int d, int r, int t, std::vector<int> *half)
{
    half->clear();
    const int R = t * r;
    auto ce = [r](int v) { return (std::abs(v) + r - 1) / r; };
    if (d == 2) {
        for (int a = -R; a <= R; a++) {
            if (shape == STENCIL_BOX) half->push_back(R);
            else half->push_back(r * (t - ce(a)));
        }
    } else {
        for (int c = -R; c <= R; c++)
            for (int a = -R; a <= R; a++) {
                if (shape == STENCIL_BOX) half->push_back(R);
                else if (ce(c) + ce(a) <= t) half->push_back(r * (t - ce(c) - ce(a)));
            }
    }
}

TcGeometry tc_geometry(int shape, int d, int r, int t, stencil_dtype dtype, int precision, int path)
{
    TcGeometry g;
    g.n_tile = 8;
    if (dtype == STENCIL_F64 && precision == STENCIL_PREC_OZAKI) {
        g.n_tile = 16;  // tcgen05 kind::f16: 16 output columns per digit block, K = 16
        g.k_inst = 16;
    } else if (dtype == STENCIL_F64) g.k_inst = 4;             // FP64 MMA m8n8k4
    else if (precision == STENCIL_PREC_BF16X3 || precision == STENCIL_PREC_F16 || precision == STENCIL_PREC_F16X3)
        g.k_inst = 16;                                         // kind::f16 K = 16
    else g.k_inst = 8;                                         // kind::tf32 K = 8
    if (d == 2 && dtype == STENCIL_F32 && (precision == STENCIL_PREC_TF32 || precision == STENCIL_PREC_TF32X3))
        g.n_tile = tc_ws_ntile(shape, r, t, precision == STENCIL_PREC_TF32X3);
    if (dtype == STENCIL_F32 &&
        (precision == STENCIL_PREC_BF16X3 || precision == STENCIL_PREC_F16 || precision == STENCIL_PREC_F16X3))
        g.n_tile = 128;  // the wide kernels: 128 output columns per MMA (their M)
    if (d == 2 && path == STENCIL_PATH_SPARSE_TENSOR_CORE) {
        // mma.sp m16n8k16: 16 output columns per block, logical K 16
        SpLayout L = sp_layout_2d(shape, r, t);
        g.n_tile = 16;
        g.k_inst = 16;
        g.kext = 4 * L.nc;
        g.sparsity = L.sparsity();
        g.available = dtype == STENCIL_F32 && precision == STENCIL_PREC_TF32 && t * r <= 12;
        return g;
    }
    if (d == 2) {
        TcLines L = tc_lines_2d(shape, r, t, g.n_tile, g.k_inst);
        g.kext = L.kext;
        g.sparsity = L.sparsity();
        g.available = t * r <= (precision == STENCIL_PREC_OZAKI ? 8 : 12);
        return g;
    }
    // 3-D: every (plane, row) line of the composite issues the K blocks of
    // its window that hold a non-zero column (R - h .. R + h + N - 1 of the
    // N + 2R columns), as tc_lines_2d counts them; the kernel exists for
    // FP32 grids in the FP16 form at t = 1 (tc3d_wide)
    std::vector<int> half;
    composite_lines(shape, d, r, t, &half);
    const int R = t * r;
    const int kext = (g.n_tile + 2 * R + g.k_inst - 1) / g.k_inst * g.k_inst, nkb = kext / g.k_inst;
    double useful = 0, issued = 0;
    for (int h : half) {
        if (h < 0) continue;
        const int lo = (R - h) / g.k_inst, hi = std::min(nkb - 1, (R + h + g.n_tile - 1) / g.k_inst);
        useful += 2 * h + 1;
        issued += (double)(hi - lo + 1) * g.k_inst;
    }
    g.kext = kext;
    g.sparsity = issued > 0 ? useful / issued : 0;
    g.available = d == 3 && dtype == STENCIL_F32 && precision == STENCIL_PREC_F16 &&
                  path == STENCIL_PATH_TENSOR_CORE && t == 1 && tc_wide3_nrows(shape, r) > 0;
    return g;
}

// Tensor-core kernels present in this build: 2-D, fused radius t*r <= 12;
// FP64 grids on the FP64 MMA, FP32 grids in the TF32 / TF32X3 / BF16X3 forms.
bool tc_supported(const Plan &p, int precision, int path)
{
    if (p.pat.d == 3)  // tc3d_wide: FP32 grids, FP16 form, one step per sweep
        return path == STENCIL_PATH_TENSOR_CORE && p.dtype == STENCIL_F32 && precision == STENCIL_PREC_F16 &&
               tc_wide3_nrows(p.pat.shape, p.pat.r) > 0;
    if (p.pat.d != 2) return false;
    if (path == STENCIL_PATH_SPARSE_TENSOR_CORE)  // mma.sp TF32 (1:2 per pair of K)
        return p.dtype == STENCIL_F32 && precision == STENCIL_PREC_TF32;
    if (path != STENCIL_PATH_TENSOR_CORE) return false;
    if (p.dtype == STENCIL_F64) return precision == STENCIL_PREC_NATIVE || precision == STENCIL_PREC_OZAKI;
    return precision == STENCIL_PREC_TF32 || precision == STENCIL_PREC_TF32X3 || precision == STENCIL_PREC_BF16X3 ||
           precision == STENCIL_PREC_F16 || precision == STENCIL_PREC_F16X3;
}

static double tc_peak(const Plan &p, int precision, int path)
{
    const stencil_peaks &pk = peaks();
    const bool sparse = path == STENCIL_PATH_SPARSE_TENSOR_CORE;
    if (p.dtype == STENCIL_F64 && precision == STENCIL_PREC_OZAKI) return pk.tc_bf16_flops;  // FP16 = BF16 rate
    if (p.dtype == STENCIL_F64) return pk.tc_f64_flops;
    if (precision == STENCIL_PREC_BF16X3 || precision == STENCIL_PREC_F16 || precision == STENCIL_PREC_F16X3)
        return sparse ? pk.sptc_bf16_flops : pk.tc_bf16_flops;  // FP16 and BF16 share the dense rate
    return sparse ? pk.sptc_tf32_flops : pk.tc_tf32_flops;
}

// Products issued per useful product: 3 for the hi/lo forms; S(S+1)/2 digit
// products (levels i + j < S of S slices each) for the exact-split FP64 form.
static double beta_of(int precision, int slices = 0)
{
    if (precision == STENCIL_PREC_OZAKI) return slices * (slices + 1) / 2.0;
    return (precision == STENCIL_PREC_TF32X3 || precision == STENCIL_PREC_BF16X3 || precision == STENCIL_PREC_F16X3)
               ? 3.0
               : 1.0;
}

// ---------------------------------------------------------------------------
// MMA-shape efficiency (the eta(N) term the paper's model does not have).
//
// On GB300 a tcgen05.mma of M = 128 and 32 bytes of K per row costs a fixed
// ~90 cycles from one instruction to the next in these kernels, whatever its
// N (16..96 measured), its operand layout or its accumulator dependencies,
// until its own arithmetic (128 N K / rate: 2048 TF32 or 4096 FP16/BF16 MACs
// per cycle) is longer.  A sweep kernel therefore runs at
//     cycles per output = max(MMAs per output * cost per MMA,
//                             worker cycles per output)
// (their sum for the wide FP16 / BF16 kernel, whose staging and epilogue
// overlap its MMAs only in part), the second term being the CUDA-core work
// of staging, rounding or cutting the input and draining the accumulators,
// measured per kernel on GB300 at 2070 MHz.  The
// instruction roof t * SMs * clock / cycles per output caps the paper's
// tensor-core roof (Eq. 12) for the dispatcher.
// ---------------------------------------------------------------------------
constexpr double kMmaCycles = 90.0;        // per tcgen05.mma, M = 128, N <= ~176
constexpr double kWorkerTf32 = 1.30;       // tc2d_ws TF32: in-place rounding, staging, epilogue
constexpr double kWorkerTf32x3 = 1.65;     // tc2d_ws TF32x3: + the lo split
constexpr double kWorkerWide = 0.45;       // tc2d_wide, one product: loads, conversion, epilogue (added to the MMAs)
constexpr double kWorkerWideSplit = 0.28;  // tc2d_wide, three products (128-row tiles, one or two buffers)
constexpr double kWorkerWide3 = 0.78;      // tc3d_wide, 128-row tiles: plane staging, strips, epilogue, runs
constexpr double kWorkerSplit = 4.06;      // tc2d_split: FP64 load, exponent, digit cut, recombination
// sptc2d_sweep issues warp-level mma.sp between its staging and epilogue
// work, so the two add: 0.92 cycles per output plus 3.15 per sparse
// instruction of an output (fitted to Box-2D2R at t = 1..4 within 4 %)
constexpr double kWorkerSparse = 0.92;
constexpr double kSparseMmaCycles = 3.15;
// cu2d_sweep FP32 (one sub-step, fixed-strip form): one FMA per tap plus
// ~19 other thread instructions per output (44 for the 25 taps of Box-2D2R,
// ncu), issued at 53.5 % of the SM's 128 per cycle; fused sub-steps repeat it
// over the overlapped tile.  Its one-step sweep saturates at ~58 % of the
// HBM roof (490 / 457 GStencil/s for Box- / Star-2D2R on 16384^2).
constexpr double kCuF32InstrPerOut = 19.0;
constexpr double kCuF32IssueEff = 0.535;
constexpr double kCuF32HbmEff = 0.58;

// Instruction-level roof (point updates/s / 1e9) of a tensor-core candidate;
// 0 when it does not apply (FP64 MMA, which the paper's model covers).
static double tc_instr_gstencils(const Plan &p, int prec, int path, int t)
{
    const stencil_peaks pk = peaks();
    const double sm_clk = pk.cu_f32_flops / 256.0;  // SMs x clock (128 FP32 FMA lanes per SM)
    if (sm_clk <= 0) return 0;
    const int shape = p.pat.shape, r = p.pat.r;
    double per_out = 0;
    if (p.pat.d == 3) {
        // tc3d_wide: per output plane tile of 128 columns x nr rows, one MMA
        // per (line, K block), plus the staging, strips and epilogue
        const int nr = tc_wide3_nrows(shape, r);
        if (p.dtype != STENCIL_F32 || prec != STENCIL_PREC_F16 || t != 1 || nr == 0) return 0;
        std::vector<int> half;
        composite_lines(shape, 3, r, 1, &half);
        const int nkb = (128 + 2 * r + 15) / 16;
        double blocks = 0;
        for (int h : half)
            if (h >= 0) blocks += std::min(nkb - 1, (r + h + 127) / 16) - (r - h) / 16 + 1;
        const double mma = blocks / (128.0 * nr) * std::max(kMmaCycles, 128.0 * nr * 16 / 4096.0);
        // the per-plane work of a tile (staging its nr + 2r rows, the strips,
        // the exchanges) is spread over nr rows of outputs
        per_out = mma + kWorkerWide3 * 128.0 / nr;
        return sm_clk / per_out / 1e9;
    }
    if (p.pat.d != 2) return 0;
    if (path == STENCIL_PATH_SPARSE_TENSOR_CORE) {
        const SpLayout L = sp_layout_2d(shape, r, t);
        double instr = 0;
        for (int m : L.mask) instr += __builtin_popcount((unsigned)m);
        per_out = kWorkerSparse + instr / (16.0 * 8.0) * kSparseMmaCycles;
    } else if (p.dtype == STENCIL_F64 && prec == STENCIL_PREC_OZAKI) {
        const int S = split_slices(p, t);
        if (S == 0) return 0;
        const TcLines L = tc_lines_2d(shape, r, t, 16, 16);
        double blocks = 0;
        for (size_t a = 0; a < L.kb_lo.size(); a++) blocks += std::max(0, L.kb_hi[a] - L.kb_lo[a] + 1);
        const double mma = blocks * S / (128.0 * 16.0) * kMmaCycles;
        per_out = std::max(mma, kWorkerSplit);
    } else if (p.dtype == STENCIL_F32 &&
               (prec == STENCIL_PREC_F16 || prec == STENCIL_PREC_F16X3 || prec == STENCIL_PREC_BF16X3) &&
               tc_wide_nrows(r, t, prec != STENCIL_PREC_F16) > 0) {
        // tc2d_wide: per tile of 128 columns x nr rows, one MMA (M = 128,
        // N = nr, K = 16) per (line, K block) and product, each costing
        // max(kMmaCycles, its arithmetic at 4096 FP16 MACs per cycle)
        const int nr = tc_wide_nrows(r, t, prec != STENCIL_PREC_F16);
        const TcLines L = tc_lines_2d(shape, r, t, 128, 16);
        double blocks = 0;
        for (size_t a = 0; a < L.kb_lo.size(); a++) blocks += std::max(0, L.kb_hi[a] - L.kb_lo[a] + 1);
        const double products = prec == STENCIL_PREC_F16 ? 1.0 : 3.0;
        const double mma = blocks * products / (128.0 * nr) * std::max(kMmaCycles, 128.0 * nr * 16 / 4096.0);
        // measured: the staging and epilogue overlap the MMAs only in part
        per_out = mma + (prec == STENCIL_PREC_F16 ? kWorkerWide : kWorkerWideSplit);
    } else if (p.dtype == STENCIL_F32 && (prec == STENCIL_PREC_TF32 || prec == STENCIL_PREC_TF32X3)) {
        const int n = tc_ws_ntile(shape, r, t, prec == STENCIL_PREC_TF32X3);
        const TcLines L = tc_lines_2d(shape, r, t, n, 8);
        double blocks = 0;
        for (size_t a = 0; a < L.kb_lo.size(); a++) blocks += std::max(0, L.kb_hi[a] - L.kb_lo[a] + 1);
        const double products = prec == STENCIL_PREC_TF32 ? 1.0 : 3.0;
        const double cost = std::max(kMmaCycles, 128.0 * n * 8 / 2048.0);
        const double mma = blocks * products / (128.0 * n) * cost;
        per_out = std::max(mma, prec == STENCIL_PREC_TF32 ? kWorkerTf32 : kWorkerTf32x3);
    } else {
        return 0;
    }
    return t * sm_clk / per_out / 1e9;
}

// CUDA-core prediction (point updates/s / 1e9) of a plan at depth t with
// output tile `tile`: min(P_CU / (2K) / overlap, t B / (2D)) (Eq. 8, with the
// redundant work of overlapped temporal tiles), and for 2-D FP32 the issue
// roof of the FP32 sub-step.
static double cu_gstencils(const Plan &p, int t, const int tile[3])
{
    const stencil_peaks pk = peaks();
    const int D = (int)p.elem_bytes();
    const double P_cu = p.dtype == STENCIL_F64 ? pk.cu_f64_flops : pk.cu_f32_flops;
    const int K = pattern_points(p.pat.shape, p.pat.d, p.pat.r);
    const double ovl = cu_overlap_factor(p, t, tile);
    double g = std::min(P_cu / (2.0 * K) / ovl, t * pk.hbm_bytes_per_s / (2.0 * D)) / 1e9;
    if (p.dtype == STENCIL_F32 && p.pat.d == 2) {
        const double per_out = ovl * t * (K + kCuF32InstrPerOut) / (128.0 * kCuF32IssueEff);
        g = std::min(g, t * (pk.cu_f32_flops / 256.0) / per_out / 1e9);
        g = std::min(g, t * kCuF32HbmEff * pk.hbm_bytes_per_s / (2.0 * D) / 1e9);
    }
    return g;
}

struct Cand {
    int path, prec, t;
    double gst;
    int tile[3];
};

static stencil_status enumerate(Plan *p, std::vector<Cand> *out);

stencil_status dispatch_candidates(Plan *p, std::vector<int> *paths, std::vector<int> *precs, std::vector<int> *ts,
                                   std::vector<double> *model)
{
    std::vector<Cand> c;
    stencil_status s = enumerate(p, &c);
    if (s != STENCIL_OK) return s;
    std::stable_sort(c.begin(), c.end(), [](const Cand &a, const Cand &b) { return a.gst > b.gst; });
    for (auto &x : c) {
        paths->push_back(x.path);
        precs->push_back(x.prec);
        ts->push_back(x.t);
        model->push_back(x.gst);
    }
    return STENCIL_OK;
}

static stencil_status enumerate(Plan *p, std::vector<Cand> *out)
{
    const stencil_peaks &pk = peaks();
    const int D = (int)p->elem_bytes();
    const int shape = p->pat.shape, d = p->pat.d, r = p->pat.r;
    const double P_cu = p->dtype == STENCIL_F64 ? pk.cu_f64_flops : pk.cu_f32_flops;
    const double B = pk.hbm_bytes_per_s;

    std::vector<int> precs;
    if (p->req_precision == STENCIL_PREC_ANY) {
        precs.push_back(STENCIL_PREC_NATIVE);
        if (p->dtype == STENCIL_F32) {
            precs.push_back(STENCIL_PREC_TF32);
            precs.push_back(STENCIL_PREC_TF32X3);
            precs.push_back(STENCIL_PREC_BF16X3);
            precs.push_back(STENCIL_PREC_F16);
            precs.push_back(STENCIL_PREC_F16X3);
        } else {
            precs.push_back(STENCIL_PREC_OZAKI);
        }
    } else {
        precs.push_back(p->req_precision);
    }
    std::vector<int> paths;
    if (p->req_path == STENCIL_PATH_AUTO) {
        paths = {STENCIL_PATH_CUDA_CORE, STENCIL_PATH_TENSOR_CORE, STENCIL_PATH_SPARSE_TENSOR_CORE};
    } else {
        paths = {p->req_path};
    }

    std::vector<Cand> &cands = *out;
    cands.clear();
    for (int path : paths) {
        for (int prec : precs) {
            if (path == STENCIL_PATH_CUDA_CORE) {
                if (prec != STENCIL_PREC_NATIVE || !cu_supported(shape, d, r)) continue;
            } else {
                if (p->dtype == STENCIL_F32 && prec == STENCIL_PREC_NATIVE) continue;  // no FP32 MMA
                if (!tc_supported(*p, prec, path)) continue;
            }
            int t_lo = p->req_t ? p->req_t : 1;
            int t_hi = p->req_t ? p->req_t : max_fused_t(*p, path);
            for (int t = t_lo; t <= t_hi; t++) {
                if (path != STENCIL_PATH_CUDA_CORE && t * r > 12) continue;
                if (path != STENCIL_PATH_CUDA_CORE && d == 3 && t != 1) continue;  // tc3d_wide: t = 1
                int slices = 0;
                if (prec == STENCIL_PREC_OZAKI) {
                    if (path != STENCIL_PATH_TENSOR_CORE) continue;
                    slices = split_slices(*p, t);
                    if (slices == 0 || split_nacc(t * r, slices) == 0) continue;
                }
                Cand c{path, prec, t, 0.0, {1, 1, 1}};
                if (path == STENCIL_PATH_CUDA_CORE) {
                    if (p->req_tile[0] || p->req_tile[1] || p->req_tile[2]) {
                        for (int i = 0; i < 3; i++) c.tile[i] = p->req_tile[i] ? p->req_tile[i] : 1;
                    } else {
                        cu_default_tile(*p, t, c.tile);
                    }
                    c.gst = cu_gstencils(*p, t, c.tile);
                } else {
                    c.tile[0] = 1;
                    c.tile[1] = p->dtype == STENCIL_F64 ? 64 : 128;
                    c.tile[2] = p->dtype == STENCIL_F64 ? 64 : (prec == STENCIL_PREC_TF32 ? 64 : (prec == STENCIL_PREC_TF32X3 ? 32 : 64));
                    if (path == STENCIL_PATH_SPARSE_TENSOR_CORE) c.tile[2] = 64;
                    if (prec == STENCIL_PREC_OZAKI) {
                        c.tile[1] = 128;
                        c.tile[2] = 16 * split_nacc(t * r, slices);
                    }
                    if (d == 3) {
                        c.tile[1] = tc_wide3_nrows(shape, r);  // one plane: rows (MMA N) x 128 columns
                        c.tile[2] = 128;
                    } else if (prec == STENCIL_PREC_BF16X3 || prec == STENCIL_PREC_F16 || prec == STENCIL_PREC_F16X3) {
                        // the wide kernel: output rows (MMA N) x 128 columns
                        const int nr = tc_wide_nrows(r, t, prec != STENCIL_PREC_F16);
                        if (nr == 0) continue;  // t r > 12
                        c.tile[1] = nr;
                        c.tile[2] = 128;
                    }
                    TcGeometry g = tc_geometry(shape, d, r, t, p->dtype, prec, path);
                    ModelOut m = model_eval(shape, d, r, t, D, g.sparsity, beta_of(prec, slices), P_cu,
                                            tc_peak(*p, prec, path), B);
                    c.gst = m.gst_tc;
                    const double gi = tc_instr_gstencils(*p, prec, path, t);
                    if (gi > 0) c.gst = std::min(c.gst, gi);
                }
                cands.push_back(c);
            }
        }
    }
    if (cands.empty())
        return fail(STENCIL_ERR_UNSUPPORTED, "no kernel for this (path, precision, shape, d, r, dtype)");
    return STENCIL_OK;
}

stencil_status dispatch(Plan *p)
{
    const stencil_peaks &pk = peaks();
    const int D = (int)p->elem_bytes();
    const int shape = p->pat.shape, d = p->pat.d, r = p->pat.r;
    const double P_cu = p->dtype == STENCIL_F64 ? pk.cu_f64_flops : pk.cu_f32_flops;
    const double B = pk.hbm_bytes_per_s;
    std::vector<Cand> cands;
    stencil_status es = enumerate(p, &cands);
    if (es != STENCIL_OK) return es;
    double best = 0;
    for (auto &c : cands) best = std::max(best, c.gst);
    const Cand *pick = nullptr;
    for (auto &c : cands) {
        if (c.gst < 0.98 * best) continue;
        if (!pick) {
            pick = &c;
            continue;
        }
        auto key = [](const Cand &x) {
            return std::make_tuple(x.path == STENCIL_PATH_CUDA_CORE ? 0 : 1, x.t,
                                   x.prec == STENCIL_PREC_OZAKI ? 100.0 : beta_of(x.prec));
        };
        if (key(c) < key(*pick)) pick = &c;
    }

    p->path = pick->path;
    p->precision = pick->prec;
    p->t = pick->t;
    for (int i = 0; i < 3; i++) p->tile[i] = pick->tile[i];

    // info: the model at the chosen t for both units
    stencil_info &in = p->info;
    std::memset(&in, 0, sizeof(in));
    in.path = p->path;
    in.precision = p->precision;
    in.t = p->t;
    for (int i = 0; i < 3; i++) in.tile[i] = p->tile[i];
    const int tc_prec = p->dtype == STENCIL_F64 ? (p->precision == STENCIL_PREC_OZAKI ? STENCIL_PREC_OZAKI
                                                                                      : STENCIL_PREC_NATIVE)
                        : (p->precision == STENCIL_PREC_NATIVE ? STENCIL_PREC_TF32 : p->precision);
    const int tc_path = p->path == STENCIL_PATH_CUDA_CORE ? STENCIL_PATH_TENSOR_CORE : p->path;
    const int slices = tc_prec == STENCIL_PREC_OZAKI ? split_slices(*p, p->t) : 0;
    TcGeometry g = tc_geometry(shape, d, r, p->t, p->dtype, tc_prec, tc_path);
    ModelOut m = model_eval(shape, d, r, p->t, D, g.sparsity, beta_of(tc_prec, slices), P_cu,
                            tc_peak(*p, tc_prec, tc_path), B);
    in.K = m.K;
    in.K_fused = m.K_fused;
    in.scenario = m.scenario;
    {
        int cut[3];
        if (p->path == STENCIL_PATH_CUDA_CORE) {
            for (int i = 0; i < 3; i++) cut[i] = p->tile[i];
        } else {
            cu_default_tile(*p, p->t, cut);
        }
        in.predicted_cu_gstencils = cu_supported(shape, d, r) ? cu_gstencils(*p, p->t, cut) : 0.0;
    }
    double gtc = m.gst_tc;
    const double gi = tc_instr_gstencils(*p, tc_prec, tc_path, p->t);
    if (gi > 0) gtc = std::min(gtc, gi);
    in.predicted_tc_gstencils = tc_supported(*p, tc_prec, tc_path) ? gtc : 0.0;
    in.predicted_gstencils = pick->gst;
    if (p->path == STENCIL_PATH_CUDA_CORE) {
        in.alpha = 1.0;
        in.sparsity = 1.0;
        in.beta = 1.0;
        in.intensity = m.I_cu;
        in.ridge = m.ridge_cu;
        in.memory_bound = m.I_cu < m.ridge_cu;
    } else {
        in.alpha = m.alpha;
        in.sparsity = g.sparsity;
        in.beta = beta_of(tc_prec, slices);
        in.intensity = m.I_tc;
        in.ridge = m.ridge_tc;
        in.memory_bound = m.I_tc < m.ridge_tc;
    }
    return STENCIL_OK;
}

static bool parse_int(const char *s, long *out)
{
    if (!s || !*s) return false;
    char *end = nullptr;
    long v = std::strtol(s, &end, 10);
    if (*end != '\0') return false;
    *out = v;
    return true;
}

}  // namespace gbs

using namespace gbs;

extern "C" {

stencil_status stencil_plan_create(stencil_plan **plan, stencil_shape shape, int d, int r,
                                   const double *weights, stencil_dtype dtype, const int64_t *dims, int t)
try {
    if (!plan) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: plan is null");
    *plan = nullptr;
    if (!weights || !dims) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: weights or dims is null");
    if (shape != STENCIL_BOX && shape != STENCIL_STAR)
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: shape must be BOX or STAR");
    if (d != 2 && d != 3) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: d must be 2 or 3");
    if (r < 1 || r > 64) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: r must be in 1..64");
    if (dtype != STENCIL_F64 && dtype != STENCIL_F32)
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: dtype must be F64 or F32");
    if (t < 0 || t > kMaxT) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: t must be in 0..16");
    Plan p;
    if (!make_pattern(shape, d, r, &p.pat)) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: pattern");
    p.dtype = dtype;
    int64_t n_int = 1, n_st = 1;
    for (int i = 0; i < 3; i++) {
        p.dims[i] = 1;
        p.ext[i] = 1;
    }
    for (int i = 0; i < d; i++) {
        if (dims[i] < 1 || dims[i] > (int64_t)1 << 31)
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: every extent must be in 1..2^31");
        p.dims[3 - d + i] = dims[i];
        p.ext[3 - d + i] = dims[i] + 2 * r;
        n_int *= dims[i];
        n_st *= dims[i] + 2 * r;
        if (n_st > ((int64_t)1 << 40))
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: grid larger than 2^40 elements");
    }
    p.n_interior = n_int;
    p.n_stored = n_st;
    p.w.assign(weights, weights + p.pat.K);
    for (double x : p.w)
        if (!std::isfinite(x)) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_create: weight not finite");
    p.req_t = t;
    if (!cu_supported(shape, d, r))
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_plan_create: no CUDA-core kernel for this (shape, d, r)");
    stencil_status s = dispatch(&p);
    if (s != STENCIL_OK) return s;
    stencil_plan *out = new (std::nothrow) stencil_plan;
    if (!out) return fail(STENCIL_ERR_OOM, "stencil_plan_create: host allocation failed");
    out->p = std::move(p);
    *plan = out;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_create");
}

stencil_status stencil_plan_set_option(stencil_plan *plan, const char *key, const char *value)
try {
    if (!plan || !key || !value) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_set_option: null argument");
    Plan trial = plan->p;
    std::string k(key), v(value);
    if (k == "path") {
        if (v == "auto") trial.req_path = STENCIL_PATH_AUTO;
        else if (v == "cuda_core") trial.req_path = STENCIL_PATH_CUDA_CORE;
        else if (v == "tensor_core") trial.req_path = STENCIL_PATH_TENSOR_CORE;
        else if (v == "sparse_tensor_core") trial.req_path = STENCIL_PATH_SPARSE_TENSOR_CORE;
        else return fail(STENCIL_ERR_INVALID_ARG, "path must be auto|cuda_core|tensor_core|sparse_tensor_core");
    } else if (k == "precision") {
        if (v == "native") trial.req_precision = STENCIL_PREC_NATIVE;
        else if (v == "tf32") trial.req_precision = STENCIL_PREC_TF32;
        else if (v == "tf32x3") trial.req_precision = STENCIL_PREC_TF32X3;
        else if (v == "bf16x3") trial.req_precision = STENCIL_PREC_BF16X3;
        else if (v == "ozaki") trial.req_precision = STENCIL_PREC_OZAKI;
        else if (v == "f16") trial.req_precision = STENCIL_PREC_F16;
        else if (v == "f16x3") trial.req_precision = STENCIL_PREC_F16X3;
        else if (v == "any") trial.req_precision = STENCIL_PREC_ANY;
        else return fail(STENCIL_ERR_INVALID_ARG, "precision must be native|tf32|tf32x3|bf16x3|f16|f16x3|ozaki|any");
        if (trial.dtype == STENCIL_F64 && trial.req_precision != STENCIL_PREC_NATIVE &&
            trial.req_precision != STENCIL_PREC_ANY && trial.req_precision != STENCIL_PREC_OZAKI)
            return fail(STENCIL_ERR_INVALID_ARG, "FP64 grids take precision native, ozaki or any");
        if (trial.dtype == STENCIL_F32 && trial.req_precision == STENCIL_PREC_OZAKI)
            return fail(STENCIL_ERR_INVALID_ARG, "precision ozaki is for FP64 grids");
    } else if (k == "t") {
        long t = 0;
        if (!parse_int(value, &t) || t < 0 || t > kMaxT) return fail(STENCIL_ERR_INVALID_ARG, "t must be 0..16");
        trial.req_t = (int)t;
    } else if (k == "tile") {
        int tl[3] = {0, 0, 0};
        if (v != "0") {
            int a = 0, b = 0, c = 0;
            char extra = 0;
            int n = std::sscanf(value, "%dx%dx%d%c", &a, &b, &c, &extra);
            if (trial.pat.d == 3 && n == 3 && a > 0 && b > 0 && c > 0) {
                tl[0] = a;
                tl[1] = b;
                tl[2] = c;
            } else if (trial.pat.d == 2 && std::sscanf(value, "%dx%d%c", &a, &b, &extra) == 2 && a > 0 && b > 0) {
                tl[0] = 1;
                tl[1] = a;
                tl[2] = b;
            } else {
                return fail(STENCIL_ERR_INVALID_ARG, "tile must be TYxTX (2-D) or TZxTYxTX (3-D)");
            }
            if (tl[2] % 4 != 0 || tl[2] > 1024 || tl[1] > 1024 || tl[0] > 1024)
                return fail(STENCIL_ERR_INVALID_ARG, "tile: TX must be a multiple of 4, sides <= 1024");
        }
        for (int i = 0; i < 3; i++) trial.req_tile[i] = tl[i];
    } else if (k == "debug_unmet_wait") {
        if (v != "0" && v != "1") return fail(STENCIL_ERR_INVALID_ARG, "debug_unmet_wait must be 0 or 1");
        trial.debug_unmet_wait = v == "1";
    } else if (k == "debug_host_exception") {
        if (v == "bad_alloc") throw std::bad_alloc();
        if (v == "runtime") throw std::runtime_error("planted by debug_host_exception");
        return fail(STENCIL_ERR_INVALID_ARG, "debug_host_exception must be bad_alloc or runtime");
    } else {
        return fail(STENCIL_ERR_INVALID_ARG, "unknown option key '" + k + "'");
    }
    stencil_status s = dispatch(&trial);
    if (s != STENCIL_OK) return s;
    plan->p = std::move(trial);
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_set_option");
}

stencil_status stencil_plan_info(const stencil_plan *plan, stencil_info *info)
try {
    if (!plan || !info) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_info: null argument");
    *info = plan->p.info;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_info");
}

size_t stencil_plan_workspace_bytes(const stencil_plan *plan, int for_host_io)
try {
    if (!plan) return 0;
    return plan->p.grid_bytes() * (for_host_io ? 3 : 1);
} catch (...) {
    gbs::abi_exception("stencil_plan_workspace_bytes");
    return 0;
}

stencil_status stencil_plan_set_workspace(stencil_plan *plan, void *dev_ptr, size_t bytes)
try {
    if (!plan) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_set_workspace: plan is null");
    if (!dev_ptr && bytes > 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_set_workspace: null with bytes > 0");
    plan->p.ws = dev_ptr;
    plan->p.ws_bytes = dev_ptr ? bytes : 0;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_set_workspace");
}

stencil_status stencil_plan_tc_layout(const stencil_plan *plan, int t, stencil_tc_layout *layout, int *kb_lo,
                                      int *kb_hi, double *B)
try {
    if (!plan || !layout) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_tc_layout: null argument");
    const Plan &p = plan->p;
    if (t < 1 || t > kMaxT) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_tc_layout: t must be 1..16");
    int prec = p.dtype == STENCIL_F64 ? (p.precision == STENCIL_PREC_OZAKI ? STENCIL_PREC_OZAKI : STENCIL_PREC_NATIVE)
                                      : p.precision;
    if (p.dtype == STENCIL_F32 && prec == STENCIL_PREC_NATIVE) prec = STENCIL_PREC_TF32;
    if (!tc_supported(p, prec, STENCIL_PATH_TENSOR_CORE) || t * p.pat.r > (prec == STENCIL_PREC_OZAKI ? 8 : 12))
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_plan_tc_layout: no tensor-core kernel for this plan and t");
    TcGeometry g = tc_geometry(p.pat.shape, p.pat.d, p.pat.r, t, p.dtype, prec, STENCIL_PATH_TENSOR_CORE);
    TcLines L = tc_lines_2d(p.pat.shape, p.pat.r, t, g.n_tile, g.k_inst);
    layout->R = L.R;
    layout->n_tile = L.n_tile;
    layout->k_inst = L.k_inst;
    layout->kext = L.kext;
    layout->nkb = L.nkb;
    layout->sparsity = L.sparsity();
    const int lines = 2 * L.R + 1;
    for (int a = 0; a < lines; a++) {
        if (kb_lo) kb_lo[a] = L.kb_lo[a];
        if (kb_hi) kb_hi[a] = L.kb_hi[a];
    }
    if (B) {
        std::vector<double> wt = compose_dense(p.pat, p.w, t);
        size_t i = 0;
        for (int a = 0; a < lines; a++)
            for (int kb = 0; kb < L.nkb; kb++)
                for (int k = 0; k < L.k_inst; k++)
                    for (int n = 0; n < L.n_tile; n++) {
                        const int b = kb * L.k_inst + k - n - L.R;
                        B[i++] = (b >= -L.R && b <= L.R) ? wt[(size_t)a * lines + (b + L.R)] : 0.0;
                    }
    }
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_tc_layout");
}

stencil_status stencil_plan_sptc_layout(const stencil_plan *plan, int t, stencil_sptc_layout *layout,
                                        int *chunk_first, int *chunk_second, unsigned char *line_mask,
                                        float *values, unsigned char *select)
try {
    if (!plan || !layout) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_sptc_layout: null argument");
    const Plan &p = plan->p;
    if (t < 1 || t > kMaxT) return fail(STENCIL_ERR_INVALID_ARG, "stencil_plan_sptc_layout: t must be 1..16");
    if (p.pat.d != 2 || p.dtype != STENCIL_F32 || t * p.pat.r > 12)
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_plan_sptc_layout: no sparse kernel for this plan and t");
    const SpLayout L = sp_layout_2d(p.pat.shape, p.pat.r, t);
    layout->R = L.R;
    layout->nc = L.nc;
    layout->ns = L.ns;
    layout->sigma = L.sigma;
    layout->sparsity = L.sparsity();
    for (int i = 0; i < 2 * L.ns; i++) {
        if (chunk_first) chunk_first[i] = L.cf[i];
        if (chunk_second) chunk_second[i] = L.cs[i];
    }
    const int lines = 2 * L.R + 1;
    for (int a = 0; a < lines; a++)
        if (line_mask) line_mask[a] = (unsigned char)L.mask[a];
    if (values || select) {
        const std::vector<double> wt = compose_dense(p.pat, p.w, t);
        size_t i = 0;
        for (int a = 0; a < lines; a++)
            for (int s = 0; s < L.ns; s++)
                for (int m = 0; m < 16; m++)
                    for (int q = 0; q < 8; q++, i++) {
                        int sel = 0;
                        const float v = sp_a_value(wt.data(), L.R, L.cf, L.cs, a, s, m, q, &sel);
                        if (values) values[i] = v;
                        if (select) select[i] = (unsigned char)sel;
                    }
    }
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_plan_sptc_layout");
}

void stencil_plan_destroy(stencil_plan *plan) { delete plan; }

const char *stencil_status_string(stencil_status s)
{
    switch (s) {
    case STENCIL_OK: return "ok";
    case STENCIL_ERR_INVALID_ARG: return "invalid argument";
    case STENCIL_ERR_UNSUPPORTED: return "unsupported";
    case STENCIL_ERR_CUDA: return "CUDA error";
    case STENCIL_ERR_OOM: return "out of memory / workspace too small";
    case STENCIL_ERR_TIMEOUT: return "device wait timed out";
    case STENCIL_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char *stencil_last_error(void) { return g_last_error.c_str(); }

uint64_t stencil_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
