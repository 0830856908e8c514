// probe.cu -- measured FMA-pipe peaks (the P_CU of the paper's Table 1 for
// this GPU): independent FMA chains in registers, timed with CUDA events,
// and scaled from the SM clock the launch ran at (clock64 against the
// global nanosecond timer, read by one thread) to the device's maximum SM
// clock (on GB300 the probe runs at the maximum clock: no change).  For
// FP64 on GB300 this loop reaches 1.01 TFLOP/s (3.2 FLOP per SM cycle at
// 2070 MHz) at every occupancy, chain count and operand source tried, while
// the FP64 stencil sweep sustains 1.24 (4.0 per cycle, FP64 pipe 99 %
// active); the dispatcher's table keeps the 4 FLOP per SM cycle.
#include <cuda_runtime.h>

#include "launch.h"

namespace gbs {
namespace {

__device__ unsigned long long g_probe_sink;
__device__ long long g_probe_clk[4];  // block 0, thread 0: clock64 and the global timer (ns), before and after

// Eight CTAs of 256 threads per SM for FP32 (64 warps); four for FP64, whose
// 16 chains of doubles need 32 registers alone (eight CTAs would cap a thread
// at 32 registers and spill the chains to local memory).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 4 : 8) fma_chains(int iters, T seed)
{
    T a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = seed + (T)(threadIdx.x + j);
    const T m = (T)0.999999, c = (T)1e-7;
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    if (timer) {
        long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        g_probe_clk[0] = clock64();
        g_probe_clk[2] = ns;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] = fma(a[j], m, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += a[j];
    if (timer) {
        long long ns;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(ns));
        g_probe_clk[1] = clock64();
        g_probe_clk[3] = ns;
    }
    if (s == (T)-12345.0) g_probe_sink = 1;  // never true; keeps the chains alive
}

// One timed launch of `blocks` CTAs: *flops_per_s = its FLOP / its CUDA-event
// time x (maximum SM clock / the SM clock it ran at).
template <typename T>
stencil_status time_chains(int blocks, int iters, cudaStream_t st, double *flops_per_s)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(STENCIL_ERR_CUDA, "cudaEventCreate");
    fma_chains<T><<<blocks, 256, 0, st>>>(iters / 8, (T)0.5);  // warm-up
    note_launch();
    cudaEventRecord(e0, st);
    fma_chains<T><<<blocks, 256, 0, st>>>(iters, (T)0.5);
    note_launch();
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "probe timing");
    long long clk[4] = {0, 0, 0, 0};
    int dev = 0, khz = 0;
    err = cudaMemcpyFromSymbol(clk, g_probe_clk, sizeof(clk));
    if (err == cudaSuccess) err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    if (err != cudaSuccess) return cuda_fail(err, "probe clock");
    *flops_per_s = (double)blocks * 256.0 * iters * 16.0 * 2.0 / (ms * 1e-3);
    const double cycles = (double)(clk[1] - clk[0]), ns = (double)(clk[3] - clk[2]);
    if (cycles > 0 && ns > 0 && khz > 0) {
        const double mhz = cycles / ns * 1e3;  // the SM clock during the launch
        if (mhz > 0.25 * khz / 1e3 && mhz < 1.05 * khz / 1e3) *flops_per_s *= (khz / 1e3) / mhz;
    }
    return STENCIL_OK;
}

}  // namespace
}  // namespace gbs

using namespace gbs;

extern "C" stencil_status stencil_probe_peaks(stencil_peaks *measured, stencil_stream_t stream)
try {
    if (!measured) return fail(STENCIL_ERR_INVALID_ARG, "stencil_probe_peaks: null pointer");
    *measured = stencil_peaks{};
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "stencil_probe_peaks: device query");
    cudaStream_t st = (cudaStream_t)stream;
    // 32 (FP64) or 64 (FP32) warps per SM, 16 independent chains each; about
    // 130 ms per timed launch at the maximum clock (2 FP64 / 128 FP32 FMA
    // lanes per SM), so the launch ramp and the clock's rise are a small part
    // of the timed region
    stencil_status s = time_chains<double>(sms * 4, 1 << 15, st, &measured->cu_f64_flops);
    if (s != STENCIL_OK) return s;
    return time_chains<float>(sms * 8, 1 << 20, st, &measured->cu_f32_flops);
} catch (...) {
    return gbs::abi_exception("stencil_probe_peaks");
}
