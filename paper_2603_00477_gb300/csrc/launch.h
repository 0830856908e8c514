// launch.h -- kernel launchers of libgbstencil (host side, CUDA runtime).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gbs {

// One fused sweep of depth t on the CUDA-core path from in to out (interior
// points only; halo cells of out are left untouched).
stencil_status launch_cu_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

// One fused sweep of depth t on CUDA cores that writes only the interior
// points closer than `band` to the boundary (after a tensor-core sweep).
stencil_status launch_cu_band(const Plan &p, const void *in, void *out, int t, int band, cudaStream_t st);

// One fused sweep of depth t on the tensor-core path (FP32: tcgen05 with the
// plan's precision form; FP64: FP64 MMA), followed by the band sweep if t > 1.
stencil_status launch_tc_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

// One fused sweep of depth t on the 2:4-structured sparse tensor-core path
// (mma.sp TF32), followed by the band sweep if t > 1.
stencil_status launch_sptc_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

// One fused sweep of depth t of an FP64 grid on the FP16 tensor cores by
// exact splitting (k_split.cu), followed by the band sweep if t > 1.
stencil_status launch_split_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

// Read and clear the split kernel's own error word (part of read_device_error).
stencil_status read_split_error(int *flag);

// One fused sweep of depth t of an FP32 grid on the FP16 / BF16 tensor cores
// with wide MMAs (k_wide.cu; precision f16, f16x3 when split, bf16x3 when
// split and bf16), without the band sweep.  STENCIL_ERR_UNSUPPORTED when its
// operands do not fit (tc_wide_nrows == 0) or for BF16 without the split.
stencil_status launch_wide_sweep(const Plan &p, const void *in, void *out, int t, bool split, bool bf16,
                                 cudaStream_t st);

// Read and clear the wide kernel's own error word (part of read_device_error).
stencil_status read_wide_error(int *flag);

// One sweep (t = 1) of a 3-D FP32 grid on the FP16 tensor cores (k_wide3d.cu,
// precision f16).  STENCIL_ERR_UNSUPPORTED for t != 1 or when no tile fits
// (tc_wide3_nrows == 0).
stencil_status launch_wide3_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st);

// Read and clear the 3-D wide kernel's own error word (part of read_device_error).
stencil_status read_wide3_error(int *flag);

// Read and clear the device error word the tensor-core kernels set when a
// bounded wait runs out (1 = timed out).
stencil_status read_device_error(int *flag);

// Copy the halo cells (the fixed boundary) of `in` to `out` and, if not null,
// to `out2`.
stencil_status launch_halo_copy(const Plan &p, const void *in, void *out, void *out2, cudaStream_t st);

// The whole run of a plan (halo copy, ceil(steps/t) fused sweeps on the
// plan's path, ping-pong through ws) on `st`; what stencil_run enqueues.
stencil_status run_sweeps(Plan &p, const void *in, void *out, void *ws, size_t ws_bytes, int64_t steps,
                          cudaStream_t st);

// Raise the dynamic shared-memory limit of kernel `func` on the current
// device to at least `bytes` (once per kernel and device; thread safe).
stencil_status ensure_smem(const void *func, size_t bytes);

// Blocks of kernel `func` resident per SM of the current device with
// `threads` threads and `smem` bytes of dynamic shared memory (after
// ensure_smem); computed once per (kernel, device, threads, smem) and
// cached for the process (thread safe).
stencil_status occupancy(const void *func, int threads, size_t smem, int *blocks);

stencil_status cuda_fail(cudaError_t e, const char *what);

}  // namespace gbs
