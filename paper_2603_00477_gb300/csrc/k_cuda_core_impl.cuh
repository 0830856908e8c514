// k_cuda_core_impl.cuh -- host launchers of the CUDA-core sweeps
// (templates; instantiated in k_cu2d_*.cu and k_cu3d.cu so that the
// instantiations compile in parallel).
#pragma once

#include <algorithm>
#include <string>

#include "cu_kernels.cuh"
#include "launch.h"

namespace gbs {
namespace cuimpl {


template <typename T>
constexpr int kV = sizeof(T) == 8 ? 4 : 8;  // strip height: FP64 needs fewer accumulators
constexpr size_t kMaxSmem = 227 * 1024;

// Band ring: tiles that contain a point closer than `band` to the interior
// boundary.  Along y these are the tile rows below ceil(band/BY) and from
// floor((ny-band)/BY) on (the last tile row may be partial), likewise in x.
inline cu::Ring make_ring(int64_t ny, int64_t nx, int BY, int BX, int band)
{
    cu::Ring g{};
    g.nty = (int)((ny + BY - 1) / BY);
    g.ntx = (int)((nx + BX - 1) / BX);
    g.band = band;
    if (band <= 0) return g;
    const int top = (int)std::min<int64_t>(g.nty, (band + BY - 1) / BY);
    const int bot = g.nty - (int)(std::max<int64_t>(0, ny - band) / BY);
    const int left = (int)std::min<int64_t>(g.ntx, (band + BX - 1) / BX);
    const int right = g.ntx - (int)(std::max<int64_t>(0, nx - band) / BX);
    g.top_w = top;
    g.rows_tb = std::min(g.nty, top + bot);
    g.left_w = left;
    g.cols_lr = std::min(g.ntx, left + right);
    return g;
}

inline int64_t ring_count(const cu::Ring &g)
{
    if (g.band <= 0) return (int64_t)g.nty * g.ntx;
    return (int64_t)g.rows_tb * g.ntx + (int64_t)(g.nty - g.rows_tb) * g.cols_lr;
}

template <typename T, int SHAPE, int R>
stencil_status launch2d(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    using Wt = cu::Weights<T, cu::Taps<SHAPE, 2, R>::K>;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 2, R>::K; k++) wt.w[k] = (T)p.w[k];
    int tile[3] = {p.tile[0], p.tile[1], p.tile[2]};
    if (band > 0 || p.path != STENCIL_PATH_CUDA_CORE) cu_default_tile(p, t, tile);
    const int BY = tile[1], BX = tile[2];
    const size_t H = BY + 2 * t * R, W = BX + 2 * t * R;
    const size_t bufb = cu::buf_elems<T>((int)H, (int)W) * sizeof(T);
    // weights (FP64) + two staging buffers (+ a work buffer for t > 1)
    const size_t smem = cu::weight_smem_bytes<T, cu::Taps<SHAPE, 2, R>::K>() + bufb * (t > 1 ? 3 : 2);
    if (smem > kMaxSmem) return fail(STENCIL_ERR_UNSUPPORTED, "CUDA-core tile does not fit in shared memory");
    auto kern = cu::cu2d_sweep<T, SHAPE, R, kV<T>>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int occ_blocks = 0;
    s = occupancy((const void *)kern, cu::kThreads, smem, &occ_blocks);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cu::Ring ring = make_ring(p.dims[1], p.dims[2], BY, BX, band);
    if (sizeof(T) == 4 && band == 0 && p.ext[2] % 4 == 0 && BX % 4 == 0 &&
        reinterpret_cast<uintptr_t>(in) % 16 == 0) {
        // shift the tile grid left so that each staged window starts on a
        // 16-byte boundary (window start = R + bx BX - t R - xshift)
        ring.xshift = (int)(((int64_t)R * (1 - t) % 4 + 4) % 4);
        ring.vec16 = 1;
        ring.ntx = (int)((p.dims[2] + ring.xshift + BX - 1) / BX);
    }
    const int64_t ntiles = ring_count(ring);
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const int64_t resident = (int64_t)std::max(1, occ_blocks) * std::max(1, sms);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, resident);
    kern<<<grid, cu::kThreads, smem, st>>>((const T *)in, (T *)out, wt, p.ext[1], p.ext[2], BY, BX, t, ring,
                                           (int)ntiles);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu2d_sweep launch");
}

// 3-D, t = 1: the streaming kernel (tile 16 RPT x 64 in y, x; chunks of
// kStreamCZ planes in z).
template <typename T, int SHAPE, int R>
stencil_status launch3d_stream(const Plan &p, const void *in, void *out, cudaStream_t st)
{
    using Wt = cu::Weights<T, cu::Taps<SHAPE, 3, R>::K>;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 3, R>::K; k++) wt.w[k] = (T)p.w[k];
    const size_t smem = cu::stream_smem_bytes<T, R>(cu::Taps<SHAPE, 3, R>::K);
    if (smem > kMaxSmem) return fail(STENCIL_ERR_UNSUPPORTED, "3-D streaming tile does not fit in shared memory");
    auto kern = cu::cu3d_stream<T, SHAPE, R>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int occ = 0;
    s = occupancy((const void *)kern, cu::kThreads, smem, &occ);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int BY = 16 * cu::stream_rows_per_thread<T>(), BX = 64;
    const int64_t tz = (p.dims[0] + cu::kStreamCZ - 1) / cu::kStreamCZ, tyy = (p.dims[1] + BY - 1) / BY,
                  txx = (p.dims[2] + BX - 1) / BX;
    const int64_t items = tz * tyy * txx;
    if (items > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(items, (int64_t)std::max(1, occ) * std::max(1, sms));
    kern<<<grid, cu::kThreads, smem, st>>>((const T *)in, (T *)out, wt, p.ext[0], p.ext[1], p.ext[2], (int)txx,
                                           (int)tyy, (int)tz, (int)items);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu3d_stream launch");
}

// 3-D, t = 1, FP32: z-marching with rotating partial sums (cu3d_rot).  The
// run of output planes per work item, cz, is chosen so that the items fill
// whole rounds of the resident CTAs: the time is ~ rounds x (cz + 2R) planes.
template <int SHAPE, int R>
stencil_status launch3d_rot(const Plan &p, const void *in, void *out, cudaStream_t st)
{
    using Wt = cu::Weights<float, cu::Taps<SHAPE, 3, R>::K>;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 3, R>::K; k++) wt.w[k] = (float)p.w[k];
    const size_t smem = cu::rot_smem_bytes<SHAPE, R>();
    auto kern = cu::cu3d_rot<SHAPE, R>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int occ = 0;
    s = occupancy((const void *)kern, cu::kThreads, smem, &occ);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int BY = 16 * cu::rot_rows_per_thread<SHAPE, R>(), BX = 64, xs = R % 4;
    const int64_t nz = p.dims[0], tyy = (p.dims[1] + BY - 1) / BY, txx = (p.dims[2] + xs + BX - 1) / BX;
    const int64_t cols = tyy * txx, slots = (int64_t)std::max(1, occ) * std::max(1, sms);
    int64_t cz = nz, best = -1;
    for (int64_t m = 1; m <= std::min<int64_t>(nz, 512); m++) {
        const int64_t c = (nz + m - 1) / m, items = ((nz + c - 1) / c) * cols;
        const int64_t cost = (items + slots - 1) / slots * (c + 2 * R);
        if (best < 0 || cost < best) {
            best = cost;
            cz = c;
        }
    }
    const int64_t items = ((nz + cz - 1) / cz) * cols;
    if (items > 0x7fffffff || cz > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(items, slots);
    kern<<<grid, cu::kThreads, smem, st>>>((const float *)in, (float *)out, wt, p.ext[0], p.ext[1], p.ext[2],
                                           (int)txx, (int)tyy, (int)items, (int)cz, xs);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu3d_rot launch");
}

template <typename T, int SHAPE, int R>
stencil_status launch3d(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (t == 1) {
        // FP32 star r <= 3 and box r = 1: rotating partial sums; the rest streams
        if constexpr (sizeof(T) == 4 && ((SHAPE == 1 && R <= 3) || (SHAPE == 0 && R == 1)))
            return launch3d_rot<SHAPE, R>(p, in, out, st);
        return launch3d_stream<T, SHAPE, R>(p, in, out, st);
    }
    using Wt = cu::Weights<T, cu::Taps<SHAPE, 3, R>::K>;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 3, R>::K; k++) wt.w[k] = (T)p.w[k];
    int tile[3] = {p.tile[0], p.tile[1], p.tile[2]};
    if (p.path != STENCIL_PATH_CUDA_CORE) cu_default_tile(p, t, tile);
    const int BZ = tile[0], BY = tile[1], BX = tile[2];
    const size_t Z = BZ + 2 * t * R, H = BY + 2 * t * R, W = BX + 2 * t * R;
    const size_t smem =
        cu::weight_smem_bytes<T, cu::Taps<SHAPE, 3, R>::K>() + Z * H * W * sizeof(T) * (t > 1 ? 3 : 2);
    if (smem > kMaxSmem) return fail(STENCIL_ERR_UNSUPPORTED, "CUDA-core tile does not fit in shared memory");
    auto kern = cu::cu3d_sweep<T, SHAPE, R, kV<T>>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int occ_blocks = 0;
    s = occupancy((const void *)kern, cu::kThreads, smem, &occ_blocks);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nz = p.dims[0], ny = p.dims[1], nx = p.dims[2];
    const int64_t tx = (nx + BX - 1) / BX, ty = (ny + BY - 1) / BY, tz = (nz + BZ - 1) / BZ;
    const int64_t ntiles = tx * ty * tz;
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const int64_t resident = (int64_t)std::max(1, occ_blocks) * std::max(1, sms);
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, resident);
    kern<<<grid, cu::kThreads, smem, st>>>((const T *)in, (T *)out, wt, p.ext[0], p.ext[1], p.ext[2], BZ, BY, BX,
                                           t, (int)tx, (int)ty, (int)ntiles);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu3d_sweep launch");
}


// Launcher of one (dtype, shape) group for the radii RLO..RHI.
template <typename T, int SHAPE, int RLO, int RHI>
stencil_status launch2d_range(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    if constexpr (RLO <= RHI) {
        if (p.pat.r == RLO) return launch2d<T, SHAPE, RLO>(p, in, out, t, band, st);
        return launch2d_range<T, SHAPE, RLO + 1, RHI>(p, in, out, t, band, st);
    }
    return fail(STENCIL_ERR_UNSUPPORTED, "no CUDA-core kernel for this (shape, d, r)");
}

}  // namespace cuimpl

// One translation unit each (the large FP32 radii compile longest, so they
// are split by radius).
stencil_status launch_cu2d_f32_box_r13(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f32_box_r45(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f32_box_r6(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f32_box_r7(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f32_star_r14(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f32_star_r57(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu2d_f64(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);
stencil_status launch_cu3d(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

}  // namespace gbs
