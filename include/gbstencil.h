/*
 * gbstencil.h -- C ABI of the GB300 (sm_103a) stencil engine.
 *
 * The engine runs repeated, temporally fused star/box stencil sweeps
 * (dimensionality d in {2,3}, radius r, fusion depth t) on one GPU, on a
 * CUDA-core path (temporal blocking in shared memory/registers) or a
 * tensor-core path (the t-step composite stencil as banded Toeplitz MMA
 * tiles), and picks the path and t with the performance model of
 * arxiv 2603.00477 ("Do We Need Tensor Cores for Stencil Computations?").
 *
 * What one step computes (paper Sec. 1 and Sec. 3.2.1, the original
 * stencil problem: one FMA per neighbouring point): every
 * interior point p of the grid becomes
 *       u_{n+1}[p] = sum_{o in O} w_o * u_n[p + o],
 * where O is the box [-r, r]^d or the star (offsets with at most one non-zero
 * coordinate) and the halo cells keep their values (fixed Dirichlet
 * boundary).  O is ordered lexicographically, first axis outermost, each
 * coordinate ascending from -r, and the K weights follow that order
 * (K = (2r+1)^d for a box, 2dr+1 for a star).  The result after `steps` steps
 * does not depend on t or on the path beyond rounding.
 *
 * Grid layout (every buffer): row-major, last axis contiguous, stored
 * extents dims[i] + 2r (the interior plus a halo of width r on every side);
 * element type double (STENCIL_F64) or float (STENCIL_F32).
 *
 * Conventions for every call:
 *   - No exception crosses this boundary; every call returns a status (an
 *     unexpected C++ exception inside the library is caught at the entry
 *     point: a failed host allocation returns STENCIL_ERR_OOM, anything
 *     else STENCIL_ERR_INTERNAL).
 *   - Device pointers are CUDA device memory of the current device
 *     (allocated by the caller, e.g. through PyTorch), never freed here.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Kernels are
 *     launched on it and the call returns without synchronising; a CUDA
 *     error reported at launch gives STENCIL_ERR_CUDA, and an asynchronous
 *     fault surfaces as STENCIL_ERR_CUDA on a later call.
 *   - A plan or batch is not thread safe: use one per stream (and thread).
 *     Library-wide state (the peak table, per-kernel launch settings, the
 *     launch counter, the last-error message per thread) is.
 *   - stencil_last_error() returns a human-readable message for the last
 *     failed call of the calling thread.
 */
#ifndef GBSTENCIL_H
#define GBSTENCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *stencil_stream_t; /* == cudaStream_t */

typedef enum {
    STENCIL_OK = 0,
    STENCIL_ERR_INVALID_ARG = 1, /* a bad argument; nothing was launched */
    STENCIL_ERR_UNSUPPORTED = 2, /* valid, but no kernel for this case   */
    STENCIL_ERR_CUDA = 3,        /* a CUDA call or launch failed          */
    STENCIL_ERR_OOM = 4,         /* workspace missing or too small, or a
                                    host allocation failed                */
    STENCIL_ERR_TIMEOUT = 5,     /* a bounded device wait ran out         */
    STENCIL_ERR_INTERNAL = 6     /* an unexpected host-side exception was
                                    caught at the entry point             */
} stencil_status;

typedef enum { STENCIL_BOX = 0, STENCIL_STAR = 1 } stencil_shape;
typedef enum { STENCIL_F64 = 0, STENCIL_F32 = 1 } stencil_dtype;

/* Execution path.  CUDA_CORE: temporal fusion with intermediates kept on
 * chip (paper Sec. 3.2.2).  TENSOR_CORE: kernel fusion into the composite
 * stencil w^(t) run as dense MMA tiles (Sec. 2.2, 3.2.3).  SPARSE_TENSOR_CORE:
 * the same on 2:4 structured-sparse MMA (Sec. 4.3). */
typedef enum {
    STENCIL_PATH_AUTO = 0,
    STENCIL_PATH_CUDA_CORE = 1,
    STENCIL_PATH_TENSOR_CORE = 2,
    STENCIL_PATH_SPARSE_TENSOR_CORE = 3
} stencil_path;

/* Arithmetic of the products.  NATIVE: the grid's own type (FP64 grids:
 * FP64 FMA or FP64 MMA; FP32 grids: FP32 FMA).  TF32: one TF32 product with
 * FP32 accumulation.  TF32X3 / BF16X3: operands split into hi + lo parts,
 * three products (hi*hi + hi*lo + lo*hi) accumulated in FP32.  OZAKI (FP64
 * grids, tensor-core path): FP64 by exact splitting (the Ozaki scheme; no
 * counterpart in the paper) -- every input tile and the composite weights
 * are cut into S balanced 9- or 8-bit integer digits (S = 6 or 7; 53+
 * significant bits), the S(S+1)/2 digit products of each level run on the
 * FP16 tensor cores with exact FP32 sums, and the levels are recombined in
 * 64-bit integers: FP64 accuracy (a few units of 2^-53 per sweep,
 * normwise).  F16 / F16X3 (FP32 grids, tensor-core path): FP16 operands with
 * a power-of-two scale per staged tile (and one for the composite weights),
 * one product (F16: 11 significant bits, TF32's) or hi + lo parts with three
 * products (F16X3: 22 bits, TF32x3's), FP32 accumulation; a kind::f16 MMA
 * takes K = 16 per instruction against TF32's 8.  3-D grids take the
 * tensor-core path only as FP32 in the F16 form at t = 1 (box r <= 2, star
 * r <= 3; a power-of-two scale per staged plane tile).  ANY: the dispatcher
 * may pick any form the grid type allows. */
typedef enum {
    STENCIL_PREC_NATIVE = 0,
    STENCIL_PREC_TF32 = 1,
    STENCIL_PREC_TF32X3 = 2,
    STENCIL_PREC_BF16X3 = 3,
    STENCIL_PREC_ANY = 4,
    STENCIL_PREC_OZAKI = 5,
    STENCIL_PREC_F16 = 6,
    STENCIL_PREC_F16X3 = 7
} stencil_precision;

/* Peak rates the model uses (bytes/s and FLOP/s).  Table 1 of the paper:
 * B (bandwidth) and P per unit.  Zero fields keep their current value. */
typedef struct {
    double hbm_bytes_per_s;  /* B                                   */
    double cu_f64_flops;     /* P_CU, FP64 FMA pipe                 */
    double cu_f32_flops;     /* P_CU, FP32 FMA pipe                 */
    double tc_f64_flops;     /* P_TC, FP64 MMA                      */
    double tc_tf32_flops;    /* P_TC, dense TF32 MMA                */
    double tc_bf16_flops;    /* P_TC, dense BF16 MMA                */
    double sptc_tf32_flops;  /* P_SpTC, 2:4 sparse TF32 (dense-equivalent) */
    double sptc_bf16_flops;  /* P_SpTC, 2:4 sparse BF16 (dense-equivalent) */
} stencil_peaks;

/* What the plan decided and what the model predicts for it. */
typedef struct {
    int path;             /* stencil_path actually used                      */
    int precision;        /* stencil_precision actually used                 */
    int t;                /* fusion depth                                    */
    int tile[3];          /* output tile per CTA, slowest axis first         */
    int K;                /* points of the pattern                           */
    int K_fused;          /* K^(t), points of the composite kernel           */
    double alpha;         /* K^(t)/(tK)  (Eq. 9); 1 on the CUDA-core path    */
    double sparsity;      /* S of the MMA tiles (useful/issued); 1 on CU     */
    double beta;          /* products issued per useful product (1 or 3)     */
    double intensity;     /* FLOP/byte of the chosen path (Eq. 8 / Eq. 12)   */
    double ridge;         /* P/B of the unit that runs the path              */
    int scenario;         /* 1..4 (Sec. 4.1) of CU vs TC at this t           */
    int memory_bound;     /* 1 if the chosen path is below its ridge         */
    double predicted_gstencils;    /* point-updates/s / 1e9 at the roof      */
    double predicted_cu_gstencils; /* CU path at this t                      */
    double predicted_tc_gstencils; /* TC path at this t (0 if not available) */
} stencil_info;

/* Input and output of the bare performance model (paper Sec. 3-4). */
typedef struct {
    int shape, d, r, t;
    int dtype_bytes;   /* D */
    double sparsity;   /* S */
    double beta;       /* products per useful product */
    double P_cu, P_tc, B;
} stencil_model_in;

typedef struct {
    int K, K_fused;
    double alpha;                 /* Eq. 9                                   */
    double C_cu, C_tc, M;         /* FLOP and bytes per point and fused sweep */
    double I_cu, I_tc;            /* Eq. 8, Eq. 12                           */
    double ridge_cu, ridge_tc;
    double P_cu_actual, P_tc_actual; /* useful FLOP/s (Eq. 8, Eq. 12)        */
    double speedup;               /* P_TC,actual / P_CU,actual (Eq. 13)      */
    int scenario;                 /* 1..4 (Sec. 4.1)                         */
    int sweet_spot;               /* scenario 3, or 4 with Eq. 19 holding    */
    double gstencils_cu, gstencils_tc; /* point-updates/s / 1e9 at the roofs */
} stencil_model_out;

/* Geometry of the tensor-core Toeplitz operands for one fusion depth
 * (paper Sec. 2.2: the stencil recast as an MMA over zero-padded banded
 * matrices).  For line a (row a of the composite kernel w^(t), a = -R..R)
 * the B operand is B_a[k][n] = w^(t)[a][k - n - R] for |k - n - R| <= R,
 * else 0, k in [0, kext), n in [0, n_tile); the MMAs issue the K blocks
 * kb_lo[a]..kb_hi[a] of k_inst columns each. */
typedef struct {
    int R;          /* fused radius t*r                          */
    int n_tile;     /* MMA N: output columns per accumulator     */
    int k_inst;     /* MMA K per instruction                     */
    int kext;       /* padded K extent of one line               */
    int nkb;        /* kext / k_inst                             */
    double sparsity;/* S = useful MACs / issued MACs             */
} stencil_tc_layout;

typedef struct stencil_plan stencil_plan;

/* ---- plans ------------------------------------------------------------- */

/* Create a plan for the stencil of Sec. 3.2.1 (K = (2r+1)^d box points or
 * 2dr+1 star points), fused t steps at a time (Sec. 3.2.2 temporal fusion on
 * CUDA cores, Sec. 2.2.3 kernel fusion on tensor cores), path and t chosen
 * by the model of Secs. 3-4 (Eqs. 8-20): `shape` (d in {2,3}, r >= 1), K weights (copied;
 * lexicographic offset order), element type `dtype`, interior extents
 * dims[0..d-1] (slowest first, each >= 1) and fusion depth t (0 = let the
 * model choose, else 1..16).  Host only: no CUDA call, no device memory.
 * Defaults: path AUTO, precision NATIVE.  Errors: INVALID_ARG for a null or
 * out-of-range argument, UNSUPPORTED when no kernel covers (shape, d, r). */
stencil_status stencil_plan_create(stencil_plan **plan, stencil_shape shape, int d, int r,
                                   const double *weights, stencil_dtype dtype,
                                   const int64_t *dims, int t);

/* Set an option and re-run dispatch (paths: Sec. 3.2.2 CUDA cores, Sec.
 * 3.2.3 tensor cores, Sec. 4.3 sparse tensor cores; the split-precision forms
 * have no counterpart in the paper).  Keys and values:
 *   "path"      auto | cuda_core | tensor_core | sparse_tensor_core
 *   "precision" native | tf32 | tf32x3 | bf16x3 | f16 | f16x3 | ozaki | any
 *               (FP32 grids: native, tf32, tf32x3, bf16x3, f16, f16x3, any;
 *               FP64 grids: native, ozaki,
 *               any.  ozaki runs on the tensor-core path only, 2-D, fused
 *               radius t*r <= 8 with 9-bit digits, <= 6 with 8-bit digits)
 *   "t"         0 (model) or 1..16
 *   "tile"      "TYxTX" (2-D) or "TZxTYxTX" (3-D) output tile, "0" = default
 *   "debug_unmet_wait"  0 | 1: test hook; 1 makes every tensor-core CTA first
 *               wait ~2 ms on an mbarrier phase that never completes, take the
 *               timeout path (error word set, tile not written) and return
 *   "debug_host_exception"  bad_alloc | runtime: test hook; the call throws
 *               that C++ exception inside the library, which the entry point
 *               turns into STENCIL_ERR_OOM / STENCIL_ERR_INTERNAL
 * INVALID_ARG for an unknown key or value, UNSUPPORTED if the requested
 * path/precision has no kernel for this plan (the plan is then unchanged). */
stencil_status stencil_plan_set_option(stencil_plan *plan, const char *key, const char *value);

/* What dispatch chose, with the model's predictions (host only): alpha
 * (Eq. 9), S (Sec. 2.2.2), intensity (Eqs. 8, 11), scenario (Sec. 4.1). */
stencil_status stencil_plan_info(const stencil_plan *plan, stencil_info *info);

/* Bytes of device workspace stencil_run needs: one stored grid, used as
 * the ping-pong buffer between fused sweeps (only touched when steps > t).
 * With for_host_io != 0: what stencil_run_host needs (three grids: input,
 * output, ping-pong). */
size_t stencil_plan_workspace_bytes(const stencil_plan *plan, int for_host_io);

/* Give the plan caller-owned device workspace (e.g. a PyTorch tensor); the
 * plan keeps the pointer until replaced or destroyed and never frees it.
 * INVALID_ARG if ptr is null with bytes > 0. */
stencil_status stencil_plan_set_workspace(stencil_plan *plan, void *dev_ptr, size_t bytes);

/* The repeated sweeps themselves (Sec. 3.2.1 per step; Sec. 3.2.2 / 2.2.3
 * per fused sweep).
 * Run `steps` steps from `in` to `out` (device buffers of the stored size,
 * halo included) on `stream`.  `in` is read only; its halo defines the fixed
 * boundary and is copied to `out`.  steps = 0 copies in to out.  The run is
 * ceil(steps/t) fused sweeps, the last one shorter if t does not divide
 * steps.  INVALID_ARG if in == out, a pointer is null, or steps < 0; OOM if
 * more than one sweep is needed and no workspace was set (the plan then
 * allocates none itself).  Asynchronous: returns after enqueueing. */
stencil_status stencil_run(stencil_plan *plan, const void *in, void *out, int64_t steps,
                           stencil_stream_t stream);

/* stencil_run from host memory (no counterpart in the paper).
 * Same computation from host memory: copies host_in to the device,
 * runs, copies the result to host_out, and synchronises `stream` before
 * returning (it also waits for the sweeps before the copy back).  Needs
 * stencil_plan_workspace_bytes(plan, 1) of workspace.  Pinned host memory
 * gives full copy bandwidth.  Right before each copy the calling thread reads
 * one byte per 4 KiB page of that host buffer: on Grace-based GB300 machines
 * the copy engine reads host pages the CPU has left alone for a few seconds
 * at ~5-16 GB/s instead of ~210 GB/s, and the touch (~3 ms per GB) restores
 * the fast rate.  Both buffers must therefore be readable by the CPU. */
stencil_status stencil_run_host(stencil_plan *plan, const void *host_in, void *host_out,
                                int64_t steps, stencil_stream_t stream);

/* Page-locked host memory for stencil_run_host (a library service; no
 * counterpart in the paper).  Allocates `bytes` (rounded up to 2 MiB) of
 * zero-filled host memory aligned to 2 MiB, advised to use transparent huge
 * pages and registered with CUDA (portable, so copies from it run at full
 * speed, ~210 GB/s host to device on GB300).  The memory belongs to the
 * caller until stencil_host_free.  INVALID_ARG for a null ptr or
 * bytes == 0; OOM if the mapping fails; CUDA if the registration fails
 * (nothing is left mapped). */
stencil_status stencil_host_alloc(void **ptr, size_t bytes);

/* Release memory from stencil_host_alloc (null is a no-op); INVALID_ARG for
 * any other pointer. */
stencil_status stencil_host_free(void *ptr);

/* The zero-padded Toeplitz operands of the tensor-core path (Sec. 2.2.1-2.2.3;
 * S as in Sec. 2.2.2).
 * The tensor-core operand layout of this plan's (dtype, precision) at fusion
 * depth t (host only).  kb_lo/kb_hi receive 2R+1 ints each; B (optional)
 * receives the FP64 Toeplitz blocks in [a][kb][k][n] order,
 * (2R+1) * nkb * k_inst * n_tile doubles.  Any of kb_lo, kb_hi, B may be null.
 * UNSUPPORTED when the tensor-core path has no kernel for the plan at this t. */
stencil_status stencil_plan_tc_layout(const stencil_plan *plan, int t, stencil_tc_layout *layout, int *kb_lo,
                                      int *kb_hi, double *B);

/* stencil_run without any device allocation, for callers that may not call
 * cudaMalloc (e.g. a plugin inside an application that owns all device memory
 * through its own allocator, or a loop that cannot take the implicit
 * synchronisation an allocation may bring).  The paper has no counterpart;
 * this is a library service.  Same computation and arguments as stencil_run,
 * but the ping-pong buffer between fused sweeps is a 64 MiB static device
 * array of this library instead of the plan's workspace (each GPU that loads
 * the library holds it until the process exits).  Grids whose stored size
 * (halo included) exceeds 64 MiB are rejected with STENCIL_ERR_UNSUPPORTED
 * when the run takes more than one fused sweep (a run of at most one sweep,
 * steps <= t, uses no scratch and takes any size).  in and out must be device
 * (or managed) memory of the current device: the array used is the current
 * device's; other buffers are rejected with STENCIL_ERR_INVALID_ARG.  Outside
 * a stream capture every call looks up the array's device address on the
 * current device (so a device reset cannot leave a stale one); during a
 * capture the address of an earlier call on that device is used, so make the
 * first call on each device before any stream capture.  All calls share the
 * one array; after a call returns its contents are unspecified (nothing in
 * it needs to start at zero: every cell a sweep reads is written earlier in
 * the same call).  Calls that overlap on the GPU, from any stream or thread,
 * race on it; the library adds no ordering between streams, so a caller
 * using several streams orders the calls itself (an event or a
 * synchronisation between them). */
stencil_status stencil_run_noalloc(stencil_plan *plan, const void *in, void *out, int64_t steps,
                                   stencil_stream_t stream);

/* Operand layout of the 2:4-structured sparse tensor-core path (Sec. 4.3) at
 * fusion depth t: the Toeplitz block of each line of w^(t) is the sparse A
 * operand of mma.sp m16n8k16 TF32 (M = 16 output columns, logical K = 16,
 * one element kept per pair of logical K).  K is permuted: the 16 + 2R input
 * columns of the window are cut into 4-column chunks (nc of them) and chunk
 * pairs (first, second) at least ceil((2R+1)/4) chunks apart are formed;
 * instruction s takes chunk pairs 2s and 2s+1, its logical pair p being
 * column 4*chunk + p/2 of chunk pair 2s + (p mod 2). */
typedef struct {
    int R;           /* fused radius t*r */
    int nc;          /* 4-column chunks of the window */
    int ns;          /* sparse instructions per line (chunk pairs / 2) */
    int sigma;       /* shared-memory row swizzle of the kernel's B loads */
    double sparsity; /* S = useful MACs / logical issued MACs */
} stencil_sptc_layout;

/* The 2:4-structured (TF32: 1:2) sparse operands of Sec. 4.3.
 * The sparse layout of this plan at fusion depth t (host only; FP32 plans,
 * 2-D, t*r <= 12, else UNSUPPORTED).  chunk_first / chunk_second receive
 * 2*ns ints (-1 = a dummy chunk); line_mask receives 2R+1 bytes (bit s: line
 * issues instruction s); values / select receive the compressed A operand,
 * (2R+1) * ns * 16 * 8 entries at [(line * ns + s) * 128 + m * 8 + p]: the
 * TF32-rounded weight kept for output column m and logical pair p, and 0 if
 * it is the pair's first member, 1 if the second.  Any output may be null. */
stencil_status stencil_plan_sptc_layout(const stencil_plan *plan, int t, stencil_sptc_layout *layout,
                                        int *chunk_first, int *chunk_second, unsigned char *line_mask,
                                        float *values, unsigned char *select);

/* One autotuning measurement. */
typedef struct {
    int path, precision, t;
    double model_gstencils;     /* the dispatcher's (model) prediction */
    double measured_gstencils;  /* point-updates/s / 1e9 on the caller's buffers */
    int tile_y, tile_x;         /* the tile the candidate ran with */
} stencil_tune_result;

/* Measurement-based choice among the candidates the model of Secs. 3-4
 * ranks (the tuner itself has no counterpart in the paper).
 * Autotuner seeded by the model: runs every (path, precision, t) the plan's
 * options allow, in the model's order (2-D CUDA-core candidates also with the
 * tiles 32x256, 64x128, 64x64, 32x128 and 128x64 unless a tile was set),
 * `reps` times `steps` steps on the
 * caller's device buffers (after one warm-up run each), times them with CUDA
 * events on `stream`, and makes the fastest the plan's choice.  Uses the
 * plan's workspace like stencil_run; `out` is overwritten.  Writes up to
 * max_results rows to `results` (may be null) and the number of candidates
 * run to *n_results (may be null).  Synchronises `stream`. */
stencil_status stencil_plan_autotune(stencil_plan *plan, const void *in, void *out, int64_t steps, int reps,
                                     stencil_stream_t stream, stencil_tune_result *results, int max_results,
                                     int *n_results);

/* Release a plan (never frees caller workspace).  Null is ignored. */
void stencil_plan_destroy(stencil_plan *plan);

/* ---- batched form ------------------------------------------------------ */

/* One 2-D grid of a batch: shape, radius (1..3), interior extents and its K
 * weights (copied at creation). */
typedef struct {
    int shape;              /* STENCIL_BOX or STENCIL_STAR */
    int r;                  /* 1..3                        */
    int64_t ny, nx;         /* interior extents, >= 1      */
    const double *weights;  /* K weights, offset order     */
} stencil_grid_desc;

typedef struct stencil_batch stencil_batch;

/* The batched form: the sweeps of Sec. 3.2.2 over many grids in one
 * persistent launch (no counterpart in the paper).
 * Many independent 2-D grids of uneven size and mixed stencils, all of one
 * dtype, run together: one persistent launch whose CTAs pull (grid, tile,
 * sweep) work items from a device queue; an item of sweep s waits (bounded)
 * for every tile of sweep s-1 of its grid.  Each grid gets the CUDA-core
 * fusion depth and tile the model picks for it (t = 0) or the given t.
 * Host only.  INVALID_ARG for bad arguments, UNSUPPORTED for r > 3. */
stencil_status stencil_batch_create(stencil_batch **batch, int n, const stencil_grid_desc *grids,
                                    stencil_dtype dtype, int t);

/* Device workspace a run of `steps` steps needs: tables, work list, counters
 * and one ping-pong grid per grid that takes more than one sweep. */
size_t stencil_batch_workspace_bytes(const stencil_batch *batch, int64_t steps);

/* Caller-owned device workspace (never freed here). */
stencil_status stencil_batch_set_workspace(stencil_batch *batch, void *dev_ptr, size_t bytes);

/* The plan information (t, tile, model) of grid i. */
stencil_status stencil_batch_info(const stencil_batch *batch, int i, stencil_info *info);

/* Run `steps` steps on every grid: ins[i] / outs[i] are device buffers of
 * grid i's stored size (host arrays of n pointers).  Uploads the run's tables
 * into the workspace (synchronising `stream` once), then launches the
 * persistent kernel.  OOM if the workspace is too small. */
stencil_status stencil_batch_run(stencil_batch *batch, const void *const *ins, void *const *outs, int64_t steps,
                                 stencil_stream_t stream);

/* Same, through a CUDA graph: the first call for a given (ins, outs, steps,
 * workspace, stream) uploads the tables and captures the counter reset and
 * the persistent kernel into a graph; later identical calls only replay it.
 * `stream` must not be the legacy default stream. */
stencil_status stencil_batch_run_graph(stencil_batch *batch, const void *const *ins, void *const *outs,
                                       int64_t steps, stencil_stream_t stream);

/* Synchronise `stream` and report STENCIL_ERR_TIMEOUT if the last run gave
 * up a dependency wait (its outputs are then incomplete). */
stencil_status stencil_batch_status(stencil_batch *batch, stencil_stream_t stream);

/* Batch options:
 *   "precision"          native | tf32 | tf32x3 | bf16x3 | any: the forms the
 *                        autotuner may give FP32 grids on tensor cores
 *                        (default native: CUDA cores only)
 *   "path"               auto | cuda_core | tensor_core | sparse_tensor_core:
 *                        put every grid on this path (its model-chosen form
 *                        and t); grids on a tensor-core path run as their own
 *                        sweeps after the persistent kernel, in the same graph
 * and, with integer values:
 *   "wait_cycles"        limit of each dependency wait in SM clock cycles
 *                        (default 2^31, about one second)
 *   "debug_block_sweep"  test hook: items of this sweep (>= 1) wait on a
 *                        counter nothing increments, so the wait runs out and
 *                        the launch aborts; -1 switches it off (default). */
stencil_status stencil_batch_set_option(stencil_batch *batch, const char *key, const char *value);

/* One measured candidate of the batched autotuner. */
typedef struct {
    int cls;          /* class index (classes ordered by shape, radius, size) */
    int shape, r;     /* the class's stencil                                   */
    int size_class;   /* interior points in [4^(6+c), 4^(7+c)): side ~ 64*2^c  */
    int ngrids;       /* grids in the class                                    */
    int path, precision, t, tile_y, tile_x;
    double model_gstencils;     /* the model's prediction (class's first grid) */
    double measured_gstencils;  /* class points * steps / s / 1e9; 0 = not run */
    int chosen;                 /* 1 for the class's winner                    */
} stencil_batch_tune_result;

/* Per-shape-class tuning of the batched form, candidates ranked by the model
 * of Secs. 3-4 (no counterpart in the paper).
 * Autotuner of the batched form, seeded by the model: groups the grids into
 * shape classes (stencil shape, radius, size class), ranks each class's
 * candidates -- CUDA-core work items (t = 1..4, tiles 16x64 .. 128x128) and,
 * for size classes >= 3 when the batch precision allows (FP64 batches, or
 * FP32 with precision other than "native"), the dense and sparse
 * tensor-core paths (t = 1..4) -- by the model, measures the model's best
 * four of each path and the current choice on the class's grids alone (`reps` timed runs of
 * `steps` steps after one untimed run, CUDA events on `stream`, inputs
 * ins/outs as for stencil_batch_run; outputs are overwritten), and gives every
 * grid of the class the fastest.  Writes up to max_results rows (results may
 * be null) and their count to *n_results.  The workspace a run needs may
 * change: query stencil_batch_workspace_bytes again.  Synchronises `stream`. */
stencil_status stencil_batch_autotune(stencil_batch *batch, const void *const *ins, void *const *outs,
                                      int64_t steps, int reps, stencil_stream_t stream,
                                      stencil_batch_tune_result *results, int max_results, int *n_results);

/* Release a batch and its cached graph (never frees caller workspace).  Null
 * is ignored. */
void stencil_batch_destroy(stencil_batch *batch);

/* ---- model ------------------------------------------------------------- */

/* The paper's model for one configuration (Sec. 3.2 Eqs. 6-12, Sec. 4.1
 * Eqs. 13-19): K, K^(t), alpha, C, M, I, ridges, attainable rates,
 * scenario and sweet spot.  Pure host arithmetic.  INVALID_ARG on null
 * pointers, d outside 1..3, r < 1, t < 1, S outside (0, 1], a
 * non-positive peak or bandwidth. */
stencil_status stencil_model_predict(const stencil_model_in *in, stencil_model_out *out);

/* The roofline inputs of Sec. 3.1 (peak compute per unit and bandwidth B;
 * P_SpTC of Eq. 20).
 * Replace the process-wide peak table the dispatcher uses (zero fields
 * unchanged) / read it.  Defaults are GB300 figures.  Thread safe; plans
 * created afterwards use the new table.  INVALID_ARG (table unchanged) for
 * a null pointer or a negative, NaN or infinite field. */
stencil_status stencil_set_peaks(const stencil_peaks *peaks);
stencil_status stencil_get_peaks(stencil_peaks *peaks);

/* Measure the FP64 and FP32 FMA-pipe rates of the current device (FLOP/s,
 * independent FMA chains in registers on every SM, one launch each on
 * `stream`; synchronises `stream`): the launch's FLOP per second (CUDA
 * events) scaled from the SM clock it ran at (clock64 against the global
 * timer) to the device's maximum SM clock.  On GB300 the FP64 figure
 * (~1.01-1.06 TFLOP/s) is below the 1.24 TFLOP/s that the FP64 stencil sweep
 * itself sustains: register-only FMA chains do not reach the FP64 pipe's
 * 4 FLOP per SM cycle.  Fills cu_f64_flops and cu_f32_flops, zeroes
 * the other fields; does not change the dispatcher's table.  Takes about a
 * second. */
stencil_status stencil_probe_peaks(stencil_peaks *measured, stencil_stream_t stream);

/* ---- diagnostics ------------------------------------------------------- */

/* Synchronise `stream` and report whether a tensor-core kernel gave up a
 * bounded wait for its MMAs since the last call (STENCIL_ERR_TIMEOUT; the
 * affected outputs were not written).  Clears the flag. */
stencil_status stencil_device_status(stencil_stream_t stream);

/* Static description of a status code ("ok", "invalid argument", ...;
 * "unknown status" for other values); never null. */
const char *stencil_status_string(stencil_status s);

/* Message of the last failing call on the calling thread (thread-local,
 * valid until that thread's next failing call); "" if none. */
const char *stencil_last_error(void);

/* Kernel launches issued through this library since it was loaded, by all
 * threads (counted on the host at each launch). */
uint64_t stencil_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif
