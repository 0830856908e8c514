// k_cuda_core.cu -- instantiations and launcher of the CUDA-core sweeps
// (templates in cu_kernels.cuh).  2-D: box and star, r = 1..7.  3-D: box
// r = 1..2, star r = 1..4.  FP64 and FP32.
#include <algorithm>
#include <atomic>
#include <string>

#include "cu_kernels.cuh"
#include "launch.h"

namespace gbs {

stencil_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(STENCIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

stencil_status ensure_smem(const void *func, size_t bytes, int *cached)
{
    if (bytes <= 48 * 1024 || (int)bytes <= *cached) return STENCIL_OK;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic smem)");
    *cached = (int)bytes;
    return STENCIL_OK;
}

namespace {

constexpr int kV = 8;
constexpr size_t kMaxSmem = 227 * 1024;

template <typename T, int SHAPE, int R>
stencil_status launch2d(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    using Wt = cu::Weights<T, cu::Taps<SHAPE, 2, R>::K>;
    static int cached = 0;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 2, R>::K; k++) wt.w[k] = (T)p.w[k];
    int tile[3] = {p.tile[0], p.tile[1], p.tile[2]};
    if (band > 0 || p.path != STENCIL_PATH_CUDA_CORE) cu_default_tile(p, t, tile);
    const int BY = tile[1], BX = tile[2];
    const size_t H = BY + 2 * t * R, W = BX + 2 * t * R;
    const size_t smem = H * W * sizeof(T) * (t > 1 ? 2 : 1);
    if (smem > kMaxSmem) return fail(STENCIL_ERR_UNSUPPORTED, "CUDA-core tile does not fit in shared memory");
    auto kern = cu::cu2d_sweep<T, SHAPE, R, kV>;
    stencil_status s = ensure_smem((const void *)kern, smem, &cached);
    if (s != STENCIL_OK) return s;
    const int64_t ny = p.dims[1], nx = p.dims[2];
    const int nty = (int)((ny + BY - 1) / BY), ntx = (int)((nx + BX - 1) / BX);
    cu::Ring ring{};
    dim3 grid((unsigned)ntx, (unsigned)nty);
    if (band > 0) {
        ring.band = band;
        ring.nty = nty;
        ring.ntx = ntx;
        ring.by_w = std::min(nty, (band + BY - 1) / BY);
        ring.bx_w = std::min(ntx, (band + BX - 1) / BX);
        ring.rows_tb = std::min(nty, 2 * ring.by_w);
        ring.cols_lr = std::min(ntx, 2 * ring.bx_w);
        const int64_t count = (int64_t)ring.rows_tb * ntx + (int64_t)(nty - ring.rows_tb) * ring.cols_lr;
        grid = dim3((unsigned)count, 1);
    } else if (grid.y > 65535) {
        return fail(STENCIL_ERR_UNSUPPORTED, "grid too tall for the tile");
    }
    kern<<<grid, cu::kThreads, smem, st>>>((const T *)in, (T *)out, wt, p.ext[1], p.ext[2], BY, BX, t, ring);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu2d_sweep launch");
}

template <typename T, int SHAPE, int R>
stencil_status launch3d(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    using Wt = cu::Weights<T, cu::Taps<SHAPE, 3, R>::K>;
    static int cached = 0;
    Wt wt;
    for (int k = 0; k < cu::Taps<SHAPE, 3, R>::K; k++) wt.w[k] = (T)p.w[k];
    const int BZ = p.tile[0], BY = p.tile[1], BX = p.tile[2];
    const size_t Z = BZ + 2 * t * R, H = BY + 2 * t * R, W = BX + 2 * t * R;
    const size_t smem = Z * H * W * sizeof(T) * (t > 1 ? 2 : 1);
    if (smem > kMaxSmem) return fail(STENCIL_ERR_UNSUPPORTED, "CUDA-core tile does not fit in shared memory");
    auto kern = cu::cu3d_sweep<T, SHAPE, R, kV>;
    stencil_status s = ensure_smem((const void *)kern, smem, &cached);
    if (s != STENCIL_OK) return s;
    const int64_t nz = p.dims[0], ny = p.dims[1], nx = p.dims[2];
    const int64_t tx = (nx + BX - 1) / BX, ty = (ny + BY - 1) / BY, tz = (nz + BZ - 1) / BZ;
    if (tx * ty > 0x7fffffff || tz > 65535) return fail(STENCIL_ERR_UNSUPPORTED, "grid too large for the tile");
    dim3 grid((unsigned)(tx * ty), (unsigned)tz);
    kern<<<grid, cu::kThreads, smem, st>>>((const T *)in, (T *)out, wt, p.ext[0], p.ext[1], p.ext[2], BZ, BY, BX,
                                           t, (int)tx);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cu3d_sweep launch");
}

template <typename T>
stencil_status launch_typed(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    const int shape = p.pat.shape, r = p.pat.r;
    if (p.pat.d == 2) {
        if (shape == STENCIL_BOX) {
            switch (r) {
            case 1: return launch2d<T, 0, 1>(p, in, out, t, band, st);
            case 2: return launch2d<T, 0, 2>(p, in, out, t, band, st);
            case 3: return launch2d<T, 0, 3>(p, in, out, t, band, st);
            case 4: return launch2d<T, 0, 4>(p, in, out, t, band, st);
            case 5: return launch2d<T, 0, 5>(p, in, out, t, band, st);
            case 6: return launch2d<T, 0, 6>(p, in, out, t, band, st);
            case 7: return launch2d<T, 0, 7>(p, in, out, t, band, st);
            }
        } else {
            switch (r) {
            case 1: return launch2d<T, 1, 1>(p, in, out, t, band, st);
            case 2: return launch2d<T, 1, 2>(p, in, out, t, band, st);
            case 3: return launch2d<T, 1, 3>(p, in, out, t, band, st);
            case 4: return launch2d<T, 1, 4>(p, in, out, t, band, st);
            case 5: return launch2d<T, 1, 5>(p, in, out, t, band, st);
            case 6: return launch2d<T, 1, 6>(p, in, out, t, band, st);
            case 7: return launch2d<T, 1, 7>(p, in, out, t, band, st);
            }
        }
    } else {
        if (shape == STENCIL_BOX) {
            switch (r) {
            case 1: return launch3d<T, 0, 1>(p, in, out, t, st);
            case 2: return launch3d<T, 0, 2>(p, in, out, t, st);
            }
        } else {
            switch (r) {
            case 1: return launch3d<T, 1, 1>(p, in, out, t, st);
            case 2: return launch3d<T, 1, 2>(p, in, out, t, st);
            case 3: return launch3d<T, 1, 3>(p, in, out, t, st);
            case 4: return launch3d<T, 1, 4>(p, in, out, t, st);
            }
        }
    }
    return fail(STENCIL_ERR_UNSUPPORTED, "no CUDA-core kernel for this (shape, d, r)");
}

}  // namespace

stencil_status launch_cu_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.dtype == STENCIL_F64) return launch_typed<double>(p, in, out, t, 0, st);
    return launch_typed<float>(p, in, out, t, 0, st);
}

stencil_status launch_cu_band(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    if (p.pat.d != 2) return fail(STENCIL_ERR_UNSUPPORTED, "band sweep: 2-D only");
    if (p.dtype == STENCIL_F64) return launch_typed<double>(p, in, out, t, band, st);
    return launch_typed<float>(p, in, out, t, band, st);
}

}  // namespace gbs
