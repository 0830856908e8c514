// k_cuda_core.cu -- dispatch of the CUDA-core sweeps (kernels in
// cu_kernels.cuh, launchers in k_cuda_core_impl.cuh, instantiated per group
// in k_cu2d_*.cu and k_cu3d.cu).
// 2-D: box and star, r = 1..7.  3-D: box r = 1..2, star r = 1..4.  FP64 and
// FP32.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>

#include "k_cuda_core_impl.cuh"

namespace gbs {

stencil_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(STENCIL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {
// Launch facts shared by every thread of the process: the dynamic
// shared-memory limit already set per (kernel, device), and resident blocks
// per SM per (kernel, device, threads, smem).  The limit only grows, and
// only under the lock, so it is never below what a launch was promised.
std::mutex g_launch_mu;
std::map<std::pair<const void *, int>, int> g_smem_limit;
std::map<std::tuple<const void *, int, int, size_t>, int> g_occupancy;
}  // namespace

stencil_status ensure_smem(const void *func, size_t bytes)
{
    if (bytes <= 48 * 1024) return STENCIL_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_launch_mu);
    int &limit = g_smem_limit[std::make_pair(func, dev)];
    if ((int)bytes <= limit) return STENCIL_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic smem)");
    limit = (int)bytes;
    return STENCIL_OK;
}

stencil_status occupancy(const void *func, int threads, size_t smem, int *blocks)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_launch_mu);
    const auto key = std::make_tuple(func, dev, threads, smem);
    auto it = g_occupancy.find(key);
    if (it == g_occupancy.end()) {
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, func, threads, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        it = g_occupancy.emplace(key, b).first;
    }
    *blocks = it->second;
    return STENCIL_OK;
}

stencil_status launch_cu_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.pat.d == 3) return launch_cu3d(p, in, out, t, st);
    if (p.pat.d != 2) return fail(STENCIL_ERR_UNSUPPORTED, "no CUDA-core kernel for this d");
    return launch_cu_band(p, in, out, t, 0, st);
}

stencil_status launch_cu_band(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st)
{
    if (p.pat.d != 2) return fail(STENCIL_ERR_UNSUPPORTED, "band sweep: 2-D only");
    if (p.dtype == STENCIL_F64) return launch_cu2d_f64(p, in, out, t, band, st);
    const int r = p.pat.r;
    if (p.pat.shape == STENCIL_BOX) {
        if (r <= 3) return launch_cu2d_f32_box_r13(p, in, out, t, band, st);
        if (r <= 5) return launch_cu2d_f32_box_r45(p, in, out, t, band, st);
        if (r == 6) return launch_cu2d_f32_box_r6(p, in, out, t, band, st);
        return launch_cu2d_f32_box_r7(p, in, out, t, band, st);
    }
    if (r <= 4) return launch_cu2d_f32_star_r14(p, in, out, t, band, st);
    return launch_cu2d_f32_star_r57(p, in, out, t, band, st);
}

}  // namespace gbs
