// run.cu -- stencil_run / stencil_run_host: the sweep schedule.
//
// A run of `steps` steps is ceil(steps / t) fused sweeps of depth t (the
// last one shorter when t does not divide steps).  Sweep k reads the output
// of sweep k-1 (the first reads `in`) and the buffers alternate between
// `out` and the workspace so that the last sweep lands in `out`; `in` is
// never written.  The fixed halo of `in` is copied once to every buffer
// that a sweep writes, because sweeps only write interior points.
#include <string>
#include <vector>

#include "launch.h"

namespace gbs {

namespace {

template <typename T>
__global__ void halo_copy_kernel(const T *__restrict__ in, T *__restrict__ out, T *__restrict__ out2, int64_t Ez,
                                 int64_t Ey, int64_t Ex, int R, int zhalo)
{
    // one warp per stored row (z, y); halo rows are copied whole, interior
    // rows only at their R cells on each end
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < Ez * Ey; row += warps) {
        const int64_t z = row / Ey, y = row % Ey;
        const bool halo_row = y < R || y >= Ey - R || (zhalo && (z < R || z >= Ez - R));
        const int64_t base = row * Ex;
        if (halo_row) {
            for (int64_t x = lane; x < Ex; x += 32) {
                T v = in[base + x];
                out[base + x] = v;
                if (out2) out2[base + x] = v;
            }
        } else {
            for (int64_t i = lane; i < 2 * R; i += 32) {
                const int64_t x = i < R ? i : Ex - 2 * R + i;
                T v = in[base + x];
                out[base + x] = v;
                if (out2) out2[base + x] = v;
            }
        }
    }
}

}  // namespace

stencil_status launch_halo_copy(const Plan &p, const void *in, void *out, void *out2, cudaStream_t st)
{
    const int R = p.pat.r;
    const int64_t rows = p.ext[0] * p.ext[1];
    int64_t blocks = (rows + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (p.dtype == STENCIL_F64)
        halo_copy_kernel<double><<<(unsigned)blocks, 256, 0, st>>>((const double *)in, (double *)out,
                                                                   (double *)out2, p.ext[0], p.ext[1], p.ext[2],
                                                                   R, p.pat.d == 3);
    else
        halo_copy_kernel<float><<<(unsigned)blocks, 256, 0, st>>>((const float *)in, (float *)out, (float *)out2,
                                                                  p.ext[0], p.ext[1], p.ext[2], R,
                                                                  p.pat.d == 3);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "halo_copy launch");
}

stencil_status run_sweeps(Plan &p, const void *in, void *out, void *ws, size_t ws_bytes, int64_t steps,
                                 cudaStream_t st)
{
    if (steps == 0) {
        cudaError_t e = cudaMemcpyAsync(out, in, p.grid_bytes(), cudaMemcpyDeviceToDevice, st);
        return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaMemcpyAsync(in -> out)");
    }
    const int t = p.t;
    const int64_t nfull = steps / t;
    const int rem = (int)(steps % t);
    const int64_t nsweeps = nfull + (rem ? 1 : 0);
    if (nsweeps > 1) {
        if (!ws || ws_bytes < p.grid_bytes())
            return fail(STENCIL_ERR_OOM, "stencil_run: more than one sweep needs a workspace of one grid "
                                         "(stencil_plan_set_workspace)");
        const char *a = (const char *)ws, *b = (const char *)in, *c = (const char *)out;
        const size_t g = p.grid_bytes();
        if ((a < b + g && b < a + g) || (a < c + g && c < a + g))
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_run: workspace overlaps in or out");
    }
    stencil_status s = launch_halo_copy(p, in, out, nsweeps > 1 ? ws : nullptr, st);
    if (s != STENCIL_OK) return s;
    const void *src = in;
    for (int64_t k = 0; k < nsweeps; k++) {
        void *dst = ((nsweeps - 1 - k) % 2 == 0) ? out : ws;
        const int tk = (k == nsweeps - 1 && rem) ? rem : t;
        if (p.path == STENCIL_PATH_CUDA_CORE) {
            s = launch_cu_sweep(p, src, dst, tk, st);
        } else if (p.path == STENCIL_PATH_TENSOR_CORE) {
            s = launch_tc_sweep(p, src, dst, tk, st);
        } else {
            s = launch_sptc_sweep(p, src, dst, tk, st);
        }
        if (s != STENCIL_OK) return s;
        src = dst;
    }
    return STENCIL_OK;
}

}  // namespace gbs

using namespace gbs;

extern "C" stencil_status stencil_run(stencil_plan *plan, const void *in, void *out, int64_t steps,
                                      stencil_stream_t stream)
try {
    if (!plan || !in || !out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run: null argument");
    if (in == out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run: in and out must differ");
    if (steps < 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run: steps < 0");
    Plan &p = plan->p;
    {
        const char *b = (const char *)in, *c = (const char *)out;
        const size_t g = p.grid_bytes();
        if (b < c + g && c < b + g) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run: in and out overlap");
    }
    return run_sweeps(p, in, out, p.ws, p.ws_bytes, steps, (cudaStream_t)stream);
} catch (...) {
    return gbs::abi_exception("stencil_run");
}

namespace gbs {
namespace {

// One CPU read per 4 KiB page of [p, p + bytes).  Measured on GB300
// (Grace CPU, coherent C2C link): once the CPU has left a host buffer alone
// for the seconds a long run takes, the GPU's copy engine reads it at
// 5-16 GB/s and writes it at ~25 GB/s -- with 4 KiB or 2 MiB pages, pinned
// or registered -- against ~210 / ~190 GB/s right after the CPU has touched
// each 4 KiB page (one read per 2 MiB does not help).  The touch costs ~3 ms
// of CPU time per GB.
volatile unsigned g_touch_sink;

void touch_pages(const void *p, size_t bytes)
{
    unsigned acc = 0;
    const uintptr_t end = reinterpret_cast<uintptr_t>(p) + bytes;
    for (uintptr_t a = reinterpret_cast<uintptr_t>(p); a < end; a = (a | 4095u) + 1)
        acc += *reinterpret_cast<const volatile unsigned char *>(a);
    g_touch_sink = acc;
}

}  // namespace
}  // namespace gbs

extern "C" stencil_status stencil_run_host(stencil_plan *plan, const void *host_in, void *host_out, int64_t steps,
                                           stencil_stream_t stream)
try {
    if (!plan || !host_in || !host_out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_host: null argument");
    if (steps < 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_host: steps < 0");
    Plan &p = plan->p;
    const size_t g = p.grid_bytes();
    if (!p.ws || p.ws_bytes < 3 * g)
        return fail(STENCIL_ERR_OOM, "stencil_run_host: needs a workspace of three grids");
    cudaStream_t st = (cudaStream_t)stream;
    char *d_in = (char *)p.ws, *d_out = d_in + g, *d_ws = d_in + 2 * g;
    touch_pages(host_in, g);  // right before the copy reads it
    cudaError_t e = cudaMemcpyAsync(d_in, host_in, g, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(host -> device)");
    stencil_status s = run_sweeps(p, d_in, d_out, d_ws, g, steps, st);
    if (s != STENCIL_OK) return s;
    // the output buffer is touched once the sweeps are done, right before the copy writes it
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    touch_pages(host_out, g);
    e = cudaMemcpyAsync(host_out, d_out, g, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(device -> host)");
    e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "cudaStreamSynchronize");
} catch (...) {
    return gbs::abi_exception("stencil_run_host");
}

extern "C" stencil_status stencil_device_status(stencil_stream_t stream)
try {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_device_status: stream");
    int flag = 0;
    stencil_status s = read_device_error(&flag);
    if (s != STENCIL_OK) return s;
    if (flag) return fail(STENCIL_ERR_TIMEOUT, "a tensor-core kernel's bounded wait for its MMAs ran out");
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_device_status");
}

// ---------------------------------------------------------------------------
// stencil_run_noalloc: the multi-sweep run without any device allocation.
//
// Some callers cannot call cudaMalloc: code embedded in a host application
// that owns all device memory through its own allocator and forbids direct
// CUDA allocations, or a latency-critical loop that cannot afford the
// implicit device synchronisation an allocation may cause.  For them the
// ping-pong buffer between fused sweeps lives in a fixed, statically sized
// device array of this library (every GPU that loads the library keeps it
// until the process exits).  The caller still passes `in` and `out`.
// ---------------------------------------------------------------------------
#include <mutex>

namespace gbs {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;  // 64 MiB
constexpr int kNoAllocMaxDevices = 64;

// In host code this name is only a host-side stand-in for the device array;
// kernels get the device address obtained from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices];

// The device address of the scratch array on the current device.  Outside a
// stream capture it is looked up again on every call (cheap), so that a
// device reset, which loads the module afresh, cannot leave a stale address;
// during a capture the address recorded by an earlier call on this device is
// used (the lookup may load the module, which a capture does not allow).
stencil_status noalloc_scratch(int dev, bool capturing, void **ptr)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_run_noalloc: device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!capturing) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "stencil_run_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = p;
    } else if (!g_noalloc_ptr[dev]) {
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_noalloc: the first call on a device must come before "
                                             "any stream capture");
    }
    *ptr = g_noalloc_ptr[dev];
    return STENCIL_OK;
}

// in and out must be device memory of the current device (the scratch array
// is the current device's): anything else would pair buffers of two devices.
stencil_status noalloc_check_device(const void *buf, int dev, const char *name)
{
    cudaPointerAttributes a{};
    cudaError_t e = cudaPointerGetAttributes(&a, buf);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_run_noalloc: cudaPointerGetAttributes");
    if (a.type == cudaMemoryTypeManaged) return STENCIL_OK;
    if (a.type != cudaMemoryTypeDevice || a.device != dev)
        return fail(STENCIL_ERR_INVALID_ARG, std::string("stencil_run_noalloc: ") + name +
                                                 " is not device memory of the current device");
    return STENCIL_OK;
}

}  // namespace
}  // namespace gbs

extern "C" stencil_status stencil_run_noalloc(stencil_plan *plan, const void *in, void *out, int64_t steps,
                                              stencil_stream_t stream)
try {
    if (!plan || !in || !out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_noalloc: null argument");
    if (in == out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_noalloc: in and out must differ");
    if (steps < 0) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_noalloc: steps < 0");
    Plan &p = plan->p;
    const size_t g = p.grid_bytes();
    {
        const char *b = (const char *)in, *c = (const char *)out;
        if (b < c + g && c < b + g) return fail(STENCIL_ERR_INVALID_ARG, "stencil_run_noalloc: in and out overlap");
    }
    // the scratch array is only the ping-pong buffer between fused sweeps: a
    // run of at most one sweep (steps <= t) needs none, at any grid size
    const int64_t nsweeps = steps / p.t + (steps % p.t ? 1 : 0);
    if (nsweeps > 1 && g > kNoAllocScratchBytes)
        return fail(STENCIL_ERR_UNSUPPORTED, "stencil_run_noalloc: the grid (" + std::to_string(g) +
                                                 " bytes with halo) exceeds the 64 MiB static scratch; "
                                                 "use stencil_run with a workspace");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_run_noalloc: cudaGetDevice");
    stencil_status s = noalloc_check_device(in, dev, "in");
    if (s == STENCIL_OK) s = noalloc_check_device(out, dev, "out");
    if (s != STENCIL_OK) return s;
    void *scratch = nullptr;
    if (nsweeps > 1) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "stencil_run_noalloc: cudaStreamIsCapturing");
        s = noalloc_scratch(dev, cap != cudaStreamCaptureStatusNone, &scratch);
        if (s != STENCIL_OK) return s;
    }
    return run_sweeps(p, in, out, scratch, scratch ? kNoAllocScratchBytes : 0, steps, (cudaStream_t)stream);
} catch (...) {
    return gbs::abi_exception("stencil_run_noalloc");
}
