// k_tc.cu -- tensor-core sweeps: the t-step composite stencil (kernel fusion,
// paper Sec. 2.2.3, Eq. 3) run as banded Toeplitz GEMM tiles.
//
// FP32 grids: tcgen05.mma with D in TMEM.  The MMA M axis runs over 128
// output rows, N over TN output columns per accumulator, K over the input
// window.  The input tile sits in shared memory "chunk-column major": 16-byte
// chunks of consecutive x, with the 16-byte chunks of consecutive rows
// adjacent.  Any 8 consecutive rows of one chunk column therefore form a
// canonical K-major core matrix, so the im2col operand A_a of line a is only
// a descriptor: start = chunk column of the window, row offset a; LBO = one
// chunk column (HS * 16 bytes), SBO = 8 rows (128 bytes).  No copy is made.
// B_a is the Toeplitz block of line a, built in shared memory by the CTA
// from the composite weights.
//   tc2d_ws (TF32, TF32X3): warp-specialised persistent kernel, TN = 32 (or
//     16 / 8 where the operands would not fit), double-buffered operands and
//     accumulators (below).
//
// Precision forms here: TF32 (one product of TF32-rounded operands) and
// TF32X3 (each operand split into hi + lo, three products hi*hi + hi*lo +
// lo*hi accumulated in FP32).  The FP16 / BF16 forms run on the wide kernel
// (k_wide.cu), which exchanges the roles of the two operands.
//
// FP64 grids (dmma2d_sweep): the same Toeplitz formulation on the FP64 MMA
// mma.sync.m8n8k4 (M = 8 output rows, N = 8 output columns, K = 4).
//
// All write interior points farther than (t-1) r from the boundary only:
// nearer points would need the halo re-imposed between the fused steps; the
// CUDA-core band kernel computes them stepwise.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "cu_kernels.cuh"
#include "launch.h"
#include "tc_layout.h"
#include "tc_ptx.cuh"

namespace gbs {

constexpr int kTcMaxR = 12;
constexpr int kTcMaxLines = 2 * kTcMaxR + 1;

struct TcParams {
    CUtensorMap tmap;  // tc2d_ws with tma: the input grid as a 2-D FP32 tensor, box 4 x (128 + 2R)
    double w[kTcMaxLines * kTcMaxLines];  // composite w^(t), (2R+1) x (2R+1), row-major
    unsigned char kb_lo[kTcMaxLines], kb_hi[kTcMaxLines];
    int R, rh, band, nkb, hs, nch;
    int debug_unmet;  // test hook: first wait on an mbarrier phase that never completes
    int vec16;        // tc2d_ws: stage 16-byte chunks (stored rows are 16-byte multiples)
    int xshift;       // tc2d_ws: tiles start xshift columns left of column 0 (aligned windows)
    int tma;          // tc2d_ws: stage tiles with TMA (one box per 16-byte chunk column)
    int64_t Ey, Ex;
};

__device__ int g_tc_error;

namespace tcs {

using namespace tc;

constexpr int TM = 128;
constexpr int TN = 8;
enum { P_TF32 = 0, P_TF32X3 = 1 };

// hi/lo split of a weight given in FP64: hi = round(w), lo = round(w - hi).
template <int PREC>
__device__ __forceinline__ void split_store_w(unsigned char *hi, unsigned char *lo, double w)
{
    if (PREC == P_TF32X3) {
        float h = to_tf32((float)w);
        *reinterpret_cast<float *>(hi) = h;
        *reinterpret_cast<float *>(lo) = to_tf32((float)(w - (double)h));
    } else {
        *reinterpret_cast<float *>(hi) = to_tf32((float)w);
    }
}

__device__ __forceinline__ bool outside_band(int64_t iy, int64_t ix, int64_t ny, int64_t nx, int band)
{
    return iy >= band && ix >= band && ny - 1 - iy >= band && nx - 1 - ix >= band;
}

constexpr unsigned long long kWaitCycles = 4ull << 30;  // ~2 s at 2 GHz
constexpr unsigned long long kDebugWaitCycles = 1ull << 22;  // ~2 ms: the test hook's limit

__device__ __forceinline__ bool wait_mbar_cycles(uint64_t *mbar, uint32_t phase,
                                                 unsigned long long limit = kWaitCycles)
{
    const unsigned long long t0 = clock64();
    while (!mbar_try_wait(mbar, phase)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Warp-specialised TF32 / TF32x3 sweep (persistent CTAs, 288 threads).
//
// An MMA of M=128 rows costs a fixed ~47 cycles for any N <= 64 (measured
// on GB300 for kind::tf32, K=8), so each MMA covers TN = 16 or 32 output
// columns (the Toeplitz block is TN x 8) rather than 8: four times the work
// per instruction for a lower sparsity factor S.  Warp 8 only issues MMAs;
// warps 0-7 load the next tile (cp.async straight into the chunk-column A
// layout, 16-byte copies when the stored rows allow, double-buffered) and
// round / split it; warps 0-3 also drain the accumulators of the previous
// tile (tcgen05.ld, double-buffered TMEM).  Three mbarriers per buffer pair
// hand work over: full[b] (operands of buffer b ready, 256 arrivals), done[b]
// (the MMAs reading buffer b and writing accumulator set b completed,
// tcgen05.commit), free[b] (accumulator set b read, 128 arrivals).  Every
// wait is bounded; a wait that runs out sets the abort flag and every warp
// leaves its loop.
// ---------------------------------------------------------------------------
template <int PREC, int TN_, int NACC>
__global__ void __launch_bounds__(288, 1)
    tc2d_ws(const float *__restrict__ in, float *__restrict__ out, const __grid_constant__ TcParams p, int ntiles,
            int ntx)
{
    constexpr bool SPLIT = PREC == P_TF32X3;
    constexpr int E = 4, TX = NACC * TN_;
    constexpr uint32_t kSet = NACC * TN_ * (SPLIT ? 2 : 1);
    constexpr uint32_t kCols = 2 * kSet;
    constexpr uint32_t kCorr = NACC * TN_;
    constexpr uint32_t kBlk = (TN_ / 8) * 256;  // bytes of one Toeplitz block (TN rows x 8 k)
    static_assert(kCols >= 32 && kCols <= 512 && (kCols & (kCols - 1)) == 0, "TMEM columns");

    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    int *abort_flag = reinterpret_cast<int *>(smem + 4);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 16);   // [2]
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + 32);   // [2]
    uint64_t *freeb = reinterpret_cast<uint64_t *>(smem + 48);  // [2]
    uint64_t *tmab = reinterpret_cast<uint64_t *>(smem + 64);   // [2] TMA copies of a buffer landed
    const int R = p.R, HS = p.hs, NCH = p.nch, nkb = p.nkb;
    const int lines = 2 * R + 1;
    const uint32_t a_bytes = (uint32_t)NCH * HS * 16;
    const uint32_t b_bytes = (uint32_t)lines * nkb * kBlk;
    unsigned char *B0 = smem + 128;
    unsigned char *B1 = B0 + (SPLIT ? b_bytes : 0);
    unsigned char *abase = B0 + b_bytes * (SPLIT ? 2 : 1);
    float *Ahi[2] = {reinterpret_cast<float *>(abase), reinterpret_cast<float *>(abase + a_bytes)};
    float *Alo[2] = {reinterpret_cast<float *>(abase + 2 * a_bytes), reinterpret_cast<float *>(abase + 3 * a_bytes)};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t Ey = p.Ey, Ex = p.Ex, rh = p.rh;
    const int64_t ny = Ey - 2 * rh, nx = Ex - 2 * rh;

    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    if (tid == 0) {
        *abort_flag = 0;
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 256);   // all eight worker warps
            mbar_init(&done[b], 1);
            mbar_init(&freeb[b], 128);  // the four epilogue warps
            mbar_init(&tmab[b], 1);     // thread 0's expect_tx arrival
        }
        fence_mbar_init();
    }
    // Toeplitz blocks: block (line, kb) = TN rows (n) x 8 k, K-major core
    // matrices (n-group i, k-chunk j) at i*256 + j*128
    const int bent = lines * nkb * TN_ * 8;
    for (int idx = tid; idx < bent; idx += blockDim.x) {
        const int k = idx % 8, n = (idx / 8) % TN_, blk = idx / (8 * TN_);
        const int ai = blk / nkb, kb = blk % nkb;
        const int b = kb * 8 + k - n - R;
        const double wv = (b >= -R && b <= R) ? p.w[ai * lines + (b + R)] : 0.0;
        const uint32_t off = blk * kBlk + (n / 8) * 256 + (k / E) * 128 + (n % 8) * 16 + (k % E) * 4;
        split_store_w<SPLIT ? P_TF32X3 : P_TF32>(B0 + off, B1 + off, wv);
    }
    fence_proxy_async_smem();
    fence_before_thread_sync();
    __syncthreads();
    fence_after_thread_sync();
    const uint32_t tmem = *tmem_slot;

    auto bounded_wait = [&](uint64_t *bar, uint32_t parity, unsigned long long limit) -> bool {
        const unsigned long long t0 = clock64();
        while (!mbar_try_wait(bar, parity)) {
            if (*(volatile int *)abort_flag) return false;
            if (clock64() - t0 > limit) {
                atomicExch(abort_flag, 1);
                return false;
            }
        }
        return true;
    };
    auto origin = [&](int id, int64_t *Y0, int64_t *X0) {
        *Y0 = rh + (int64_t)(id / ntx) * TM;
        *X0 = (int64_t)(id % ntx) * TX - p.xshift;
    };

    if (warp == 8) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kFmtTF32, TM, TN_);
            const uint32_t lbo_a = (uint32_t)HS * 16;
            const uint32_t b0 = smem_u32(B0), b1 = smem_u32(B1);
            int k = 0;
            for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
                const int b = k & 1;
                if (!bounded_wait(&full[b], (k >> 1) & 1, kWaitCycles)) break;
                if (k >= 2 && !bounded_wait(&freeb[b], ((k - 2) >> 1) & 1, kWaitCycles)) break;
                fence_after_thread_sync();
                // Descriptors advance by adding offsets in 16-byte units to the
                // start-address field (bits 0-13; every address < 256 KB).
                const uint64_t da_base = smem_desc(smem_u32(Ahi[b]), lbo_a, 128);
                const uint64_t db_base = smem_desc(b0, 128, 256);
                const uint64_t dlo_a = (uint64_t)((smem_u32(Alo[b]) - smem_u32(Ahi[b])) >> 4);
                const uint64_t dlo_b = (uint64_t)((b1 - b0) >> 4);
                const uint64_t kb_step_a = (uint64_t)2 * HS;   // two chunk columns
                const uint64_t blk16 = kBlk >> 4;
                const uint32_t dset = tmem + b * kSet;
                // Consecutive MMAs go to different accumulators (q innermost) and
                // share the Toeplitz block: MMAs chained on one accumulator issue
                // about 1.3x slower (measured with clock64 traces).
                uint32_t acc = 0;
                for (int ai = 0; ai < lines; ++ai) {
                    const int klo = p.kb_lo[ai], khi = p.kb_hi[ai];
                    uint64_t da = da_base + (uint64_t)ai + (uint64_t)klo * kb_step_a;
                    uint64_t db = db_base + (uint64_t)(ai * nkb + klo) * blk16;
                    for (int kb = klo; kb <= khi; ++kb) {
#pragma unroll
                        for (int q = 0; q < NACC; ++q) {
                            const uint32_t d = dset + q * TN_, dc = d + kCorr;
                            const uint64_t daq = da + (uint64_t)(q * (TN_ / E)) * HS;
                            mma_tf32(d, daq, db, idesc, acc);
                            if (SPLIT) {
                                mma_tf32(dc, daq, db + dlo_b, idesc, acc);
                                mma_tf32(dc, daq + dlo_a, db, idesc, 1);
                            }
                        }
                        acc = 1;
                        da += kb_step_a;
                        db += blk16;
                    }
                }
                mma_commit(&done[b]);
            }
            // let the last MMAs finish before TMEM can be freed (no early exit
            // on abort here: this wait protects the TMEM the MMAs write)
            if (k >= 1) wait_mbar_cycles(&done[(k - 1) & 1], ((k - 1) >> 1) & 1);
            if (k >= 2) wait_mbar_cycles(&done[(k - 2) & 1], ((k - 2) >> 1) & 1);
        }
        __syncwarp();
    } else {
        // ---------------- loaders / converters (warps 0-7), epilogue (warps 0-3) -----
        const int rows = TM + 2 * R, cols = NCH * E;
        int tma_pending = -1;  // buffer whose TMA copies may still be in flight
        auto prefetch = [&](int id, float *dst, int buf) {
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            if (p.tma) {
                // one box of 4 values x rows per 16-byte chunk column (X0 - R is a
                // multiple of 4: every box starts on a 16-byte boundary); rows and
                // chunks outside the grid arrive as zeros
                if (tid == 0) {
                    mbar_arrive_expect_tx(&tmab[buf], (uint32_t)(NCH * rows * 16));
                    for (int c = 0; c < NCH; ++c)
                        tma_load_2d(reinterpret_cast<unsigned char *>(dst) + (size_t)c * HS * 16, &p.tmap,
                                    (int)(X0 - R) + 4 * c, (int)(Y0 - R), &tmab[buf]);
                }
                tma_pending = buf;
                return;
            }
            if (p.vec16) {
                // one 16-byte copy per (row, chunk column); X0 - R is a multiple of 4,
                // so each chunk lies wholly inside or wholly outside its row
                for (int row = warp; row < rows; row += 8) {
                    const int64_t gy = Y0 - R + row;
                    const bool rowok = gy >= 0 && gy < Ey;
                    const float *grow = in + (rowok ? gy : 0) * Ex;
                    for (int c = lane; c < NCH; c += 32) {
                        const int64_t gx = X0 - R + 4 * c;
                        const bool ok = rowok && gx >= 0 && gx < Ex;
                        const uint32_t d = smem_u32(dst) + (uint32_t)(c * HS + row) * 16;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d),
                                     "l"(ok ? grow + gx : in), "r"(ok ? 16 : 0)
                                     : "memory");
                    }
                }
                return;
            }
            for (int row = warp; row < rows; row += 8) {
                const int64_t gy = Y0 - R + row;
                const bool rowok = gy >= 0 && gy < Ey;
                for (int x = lane; x < cols; x += 32) {
                    const int64_t gx = X0 - R + x;
                    const bool ok = rowok && gx >= 0 && gx < Ex;
                    cu::cp_async_elem<4>(reinterpret_cast<unsigned char *>(dst) + (x / E) * HS * 16 + row * 16 +
                                             (x % E) * 4,
                                         ok ? in + gy * Ex + gx : in, ok);
                }
            }
        };
        auto epilogue = [&](int id, uint32_t set_base) {
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            const int m = warp * 32 + lane;
            const int64_t gy = Y0 + m, iy = gy - rh;
            const bool rowok = iy < ny && iy >= p.band && ny - 1 - iy >= p.band;
            const uint32_t lane_base = set_base + ((uint32_t)(warp * 32) << 16);
            for (int q = 0; q < NACC; ++q) {
#pragma unroll
                for (int h = 0; h < TN_ / 8; ++h) {
                    uint32_t v[8], c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    tmem_ld_32x32b_x8(lane_base + q * TN_ + h * 8, v);
                    if (SPLIT) tmem_ld_32x32b_x8(lane_base + kCorr + q * TN_ + h * 8, c);
                    tmem_ld_wait();
                    if (!rowok) continue;
                    float f[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        f[j] = __uint_as_float(v[j]) + (SPLIT ? __uint_as_float(c[j]) : 0.0f);
                    const int64_t gx0 = X0 + q * TN_ + h * 8;
                    float *dst = out + gy * Ex + gx0;
                    const bool fullrow = gx0 >= rh + p.band && gx0 + 7 < Ex - rh - p.band;
                    const uintptr_t al = reinterpret_cast<uintptr_t>(dst) & 15;
                    if (fullrow && al == 0) {
                        reinterpret_cast<float4 *>(dst)[0] = make_float4(f[0], f[1], f[2], f[3]);
                        reinterpret_cast<float4 *>(dst)[1] = make_float4(f[4], f[5], f[6], f[7]);
                    } else if (fullrow && (al & 7) == 0) {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            reinterpret_cast<float2 *>(dst)[j] = make_float2(f[2 * j], f[2 * j + 1]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int64_t ix = gx0 + j - rh;
                            if (ix >= p.band && ix < nx - p.band) dst[j] = f[j];
                        }
                    }
                }
            }
        };

        int k = 0, prev = -1;
        if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x, Ahi[0], 0);
        cu::cp_async_commit();
        bool ok = true;
        for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
            const int b = k & 1;
            if (p.tma) {
                // buffer b's TMA copies have landed (phase = its use count)
                if (!bounded_wait(&tmab[b], (k >> 1) & 1, kWaitCycles)) {
                    ok = false;
                    break;
                }
                tma_pending = -1;
            } else {
                cu::cp_async_wait_group<0>();
                named_bar_sync(1, 256);
                if (*(volatile int *)abort_flag) {
                    ok = false;
                    break;
                }
            }
            // round to TF32 in place (and split off the lo part), 16 bytes at a time
            const int quads = (int)(a_bytes / 16);
            float4 *A = reinterpret_cast<float4 *>(Ahi[b]), *L = reinterpret_cast<float4 *>(Alo[b]);
            for (int i = tid; i < quads; i += 256) {
                const float4 u = A[i];
                const float4 hi = make_float4(to_tf32(u.x), to_tf32(u.y), to_tf32(u.z), to_tf32(u.w));
                A[i] = hi;
                if (SPLIT)
                    L[i] = make_float4(to_tf32(u.x - hi.x), to_tf32(u.y - hi.y), to_tf32(u.z - hi.z),
                                       to_tf32(u.w - hi.w));
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[b]);
            if (k >= 1) {  // tile k-1: its MMAs released buffer b^1 and filled accumulator set b^1
                if (!bounded_wait(&done[b ^ 1], ((k - 1) >> 1) & 1, kWaitCycles)) {
                    ok = false;
                    break;
                }
                fence_after_thread_sync();
            }
            // the next tile's loads go out first; the epilogue hides their latency
            const int nid = id + gridDim.x;
            if (nid < ntiles) prefetch(nid, Ahi[b ^ 1], b ^ 1);
            cu::cp_async_commit();
            if (k >= 1 && warp < 4) {
                epilogue(prev, tmem + (b ^ 1) * kSet);
                fence_before_thread_sync();
                mbar_arrive(&freeb[b ^ 1]);
            }
            prev = id;
        }
        if (ok && prev >= 0) {
            const int lb = (k - 1) & 1;
            ok = bounded_wait(&done[lb], ((k - 1) >> 1) & 1, kWaitCycles);
            fence_after_thread_sync();
            // test hook: the barrier's next phase is never completed
            if (ok && p.debug_unmet) ok = bounded_wait(&done[lb], (((k - 1) >> 1) & 1) ^ 1, kDebugWaitCycles);
            if (ok && warp < 4) epilogue(prev, tmem + lb * kSet);
        }
        cu::cp_async_wait_group<0>();
        if (!ok) atomicExch(abort_flag, 1);
        // after an abort, TMA copies issued for the next tile may still be in
        // flight: let them land (bounded) before the CTA's shared memory goes
        if (tma_pending >= 0 && tid == 0) {
            const unsigned long long t0 = clock64();
            while (!mbar_try_wait(&tmab[tma_pending], (k >> 1) & 1) && clock64() - t0 < kWaitCycles) {
            }
        }
    }
    fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *(volatile int *)abort_flag) atomicExch(&g_tc_error, 1);
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// FP64: mma.sync.m8n8k4 (A 8x4 row-major, B 4x8 column-major, C/D 8x8).
// 256 threads; a CTA owns 64 output rows x 64 output columns; warp w owns
// rows 8w..8w+7 and eight 8-column accumulators.
// ---------------------------------------------------------------------------
constexpr int DM_T = 64;

__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b)
{
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                 : "+d"(d0), "+d"(d1)
                 : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(256) dmma2d_sweep(const double *__restrict__ in, double *__restrict__ out,
                                                    const __grid_constant__ TcParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int R = p.R, lines = 2 * R + 1, nkb = p.nkb;  // K step 4
    const int W = DM_T + 8 * 0 + p.nch;                  // smem row length (doubles)
    const int H = DM_T + 2 * R;
    double *S = reinterpret_cast<double *>(smem_raw);
    double *Bf = S + (size_t)H * W;  // [ai][kb][lane] fragments: B[lane%4][lane/4]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t Y0 = p.rh + (int64_t)blockIdx.y * DM_T;
    const int64_t X0 = p.rh + (int64_t)blockIdx.x * DM_T;
    const int64_t ny = p.Ey - 2 * p.rh, nx = p.Ex - 2 * p.rh;

    for (int idx = tid; idx < lines * nkb * 32; idx += blockDim.x) {
        const int l = idx % 32, blk = idx / 32;
        const int ai = blk / nkb, kb = blk % nkb;
        const int k = kb * 4 + (l & 3), n = l >> 2;
        const int b = k - n - R;
        Bf[idx] = (b >= -R && b <= R) ? p.w[ai * lines + (b + R)] : 0.0;
    }
    for (int row = warp; row < H; row += 8) {
        const int64_t gy = Y0 - R + row;
        const bool rowok = gy >= 0 && gy < p.Ey;
        for (int x = lane; x < W; x += 32) {
            const int64_t gx = X0 - R + x;
            S[row * W + x] = (rowok && gx >= 0 && gx < p.Ex) ? __ldg(in + gy * p.Ex + gx) : 0.0;
        }
    }
    __syncthreads();

    const int g = lane >> 2, c = lane & 3;
    double acc[8][2];
#pragma unroll
    for (int nb = 0; nb < 8; ++nb) acc[nb][0] = acc[nb][1] = 0.0;
    for (int ai = 0; ai < lines; ++ai) {
        const double *srow = S + (warp * 8 + g + ai) * W + c;
        for (int kb = p.kb_lo[ai]; kb <= p.kb_hi[ai]; ++kb) {
            const double b = Bf[(ai * nkb + kb) * 32 + lane];
#pragma unroll
            for (int nb = 0; nb < 8; ++nb) dmma(acc[nb][0], acc[nb][1], srow[nb * 8 + kb * 4], b);
        }
    }
    const int64_t gy = Y0 + warp * 8 + g, iy = gy - p.rh;
    if (iy < ny) {
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t ix = X0 - p.rh + nb * 8 + 2 * c + h;
                if (ix < nx && outside_band(iy, ix, ny, nx, p.band)) out[gy * p.Ex + p.rh + ix] = acc[nb][h];
            }
        }
    }
}

}  // namespace tcs

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

stencil_status fill_params(const Plan &p, int t, int n_tile, int k_inst, TcParams *tp, TcLines *L)
{
    const int r = p.pat.r, R = t * r;
    if (R > kTcMaxR) return fail(STENCIL_ERR_UNSUPPORTED, "tensor-core path: fused radius t*r must be <= 12");
    *L = tc_lines_2d(p.pat.shape, r, t, n_tile, k_inst);
    std::vector<double> wt = compose_dense(p.pat, p.w, t);
    std::memset(tp, 0, sizeof(*tp));
    const int lines = 2 * R + 1;
    for (int i = 0; i < lines * lines; i++) tp->w[i] = wt[i];
    for (int a = 0; a < lines; a++) {
        tp->kb_lo[a] = (unsigned char)L->kb_lo[a];
        tp->kb_hi[a] = (unsigned char)L->kb_hi[a];
        if (L->kb_lo[a] > L->kb_hi[a]) {  // empty line
            tp->kb_lo[a] = 1;
            tp->kb_hi[a] = 0;
        }
    }
    tp->R = R;
    tp->rh = r;
    tp->debug_unmet = p.debug_unmet_wait;
    tp->band = (t - 1) * r;
    tp->nkb = L->nkb;
    tp->Ey = p.ext[1];
    tp->Ex = p.ext[2];
    return STENCIL_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (the library links only the runtime); null if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// The FP32 input grid (Ey rows of Ex values, row pitch Ex * 4 bytes) as a 2-D
// tensor map whose box is one 16-byte chunk column of a staged tile: 4 values
// x rows.  Out-of-range elements load as zeros.  False if the map cannot be
// made (the kernel then stages with cp.async).
bool make_chunk_column_map(CUtensorMap *m, const void *in, int64_t Ey, int64_t Ex, int rows)
{
    EncodeTiledFn enc = encode_tiled();
    if (!enc || rows > 256) return false;
    const cuuint64_t dim[2] = {(cuuint64_t)Ex, (cuuint64_t)Ey};
    const cuuint64_t stride[1] = {(cuuint64_t)Ex * 4};
    const cuuint32_t box[2] = {4, (cuuint32_t)rows};
    const cuuint32_t estride[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(in), dim, stride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int PREC, int TN_, int NACC>
stencil_status launch_tc2d_ws_n(const Plan &p, const void *in, void *out, int t, cudaStream_t st, bool *fits)
{
    using namespace tcs;
    constexpr int TX = NACC * TN_;
    TcParams tp;
    TcLines L;
    stencil_status s = fill_params(p, t, TN_, 8, &tp, &L);
    if (s != STENCIL_OK) return s;
    const int R = tp.R;
    tp.hs = (TM + 2 * R + 7) / 8 * 8;  // chunk columns 128-byte aligned (TMA destinations)
    tp.nch = (TN_ * (NACC - 1) + L.kext) / 4;
    const bool split = PREC == P_TF32X3;
    const size_t a_bytes = (size_t)tp.nch * tp.hs * 16;
    const size_t b_bytes = (size_t)(2 * R + 1) * L.nkb * (TN_ / 8) * 256;
    const size_t smem = 128 + b_bytes * (split ? 2 : 1) + a_bytes * (split ? 4 : 2);
    *fits = smem <= 227 * 1024;
    if (!*fits) return STENCIL_OK;
    auto kern = tc2d_ws<PREC, TN_, NACC>;
    s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 16-byte staging when every stored row is a 16-byte multiple: the tile
    // grid then starts xshift columns left of column 0 so that each staged
    // window (tile start - R) begins on a 16-byte boundary
    tp.vec16 = (p.ext[2] % 4 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
    tp.xshift = tp.vec16 ? (4 - R % 4) % 4 : 0;
    // TMA staging needs 16-byte rows and aligned windows (vec16)
    tp.tma = tp.vec16 && make_chunk_column_map(&tp.tmap, in, p.ext[1], p.ext[2], TM + 2 * R);
    const int64_t nty = (p.dims[1] + TM - 1) / TM, ntx = (p.ext[2] + tp.xshift + TX - 1) / TX;
    const int64_t ntiles = nty * ntx;
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
    kern<<<grid, 288, smem, st>>>((const float *)in, (float *)out, tp, (int)ntiles, (int)ntx);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "tc2d_ws launch");
}

// Widest MMA N whose operands fit in shared memory (the rule the dispatcher
// uses to report S, tc_ws_ntile).
template <int PREC>
stencil_status launch_tc2d_ws(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    bool fits = false;
    const int tn = tc_ws_ntile(p.pat.shape, p.pat.r, t, PREC == tcs::P_TF32X3);
    stencil_status s;
    if (tn == 32) s = launch_tc2d_ws_n<PREC, 32, 2>(p, in, out, t, st, &fits);
    else if (tn == 16) s = launch_tc2d_ws_n<PREC, 16, 2>(p, in, out, t, st, &fits);
    else s = launch_tc2d_ws_n<PREC, 8, 4>(p, in, out, t, st, &fits);
    if (s != STENCIL_OK) return s;
    return fits ? STENCIL_OK : fail(STENCIL_ERR_UNSUPPORTED, "tensor-core tile does not fit in shared memory");
}

stencil_status launch_dmma2d(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    using namespace tcs;
    TcParams tp;
    TcLines L;
    stencil_status s = fill_params(p, t, 8, 4, &tp, &L);
    if (s != STENCIL_OK) return s;
    const int R = tp.R;
    // smem row: the widest window read is 8*7 + kext columns
    tp.nch = 8 * 7 + L.kext - DM_T;  // extra columns beyond DM_T
    if (tp.nch < 0) tp.nch = 0;
    const int W = DM_T + tp.nch, H = DM_T + 2 * R;
    const size_t smem = ((size_t)H * W + (size_t)(2 * R + 1) * L.nkb * 32) * 8;
    if (smem > 227 * 1024) return fail(STENCIL_ERR_UNSUPPORTED, "FP64 MMA tile does not fit in shared memory");
    s = ensure_smem((const void *)dmma2d_sweep, smem);
    if (s != STENCIL_OK) return s;
    const int64_t ny = p.dims[1], nx = p.dims[2];
    dim3 grid((unsigned)((nx + DM_T - 1) / DM_T), (unsigned)((ny + DM_T - 1) / DM_T));
    dmma2d_sweep<<<grid, 256, smem, st>>>((const double *)in, (double *)out, tp);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "dmma2d_sweep launch");
}

}  // namespace

stencil_status launch_tc_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.pat.d == 3 && p.dtype == STENCIL_F32 && p.precision == STENCIL_PREC_F16)
        return launch_wide3_sweep(p, in, out, t, st);  // t = 1: no band
    if (p.pat.d != 2) return fail(STENCIL_ERR_UNSUPPORTED, "tensor-core path: 3-D grids in FP32 with precision f16 only");
    stencil_status s;
    if (p.dtype == STENCIL_F64 && p.precision == STENCIL_PREC_OZAKI) {
        return launch_split_sweep(p, in, out, t, st);  // includes the band sweep
    } else if (p.dtype == STENCIL_F64) {
        s = launch_dmma2d(p, in, out, t, st);
    } else {
        switch (p.precision) {
        case STENCIL_PREC_TF32: s = launch_tc2d_ws<tcs::P_TF32>(p, in, out, t, st); break;
        case STENCIL_PREC_TF32X3: s = launch_tc2d_ws<tcs::P_TF32X3>(p, in, out, t, st); break;
        // the FP16 / BF16 forms: the wide kernel (a tile fits for every t r <= 12)
        case STENCIL_PREC_BF16X3: s = launch_wide_sweep(p, in, out, t, true, true, st); break;
        case STENCIL_PREC_F16: s = launch_wide_sweep(p, in, out, t, false, false, st); break;
        case STENCIL_PREC_F16X3: s = launch_wide_sweep(p, in, out, t, true, false, st); break;
        default: return fail(STENCIL_ERR_UNSUPPORTED, "tensor-core path: precision");
        }
    }
    if (s != STENCIL_OK || t == 1) return s;
    // points within (t-1) r of the boundary: stepwise on CUDA cores
    return launch_cu_band(p, in, out, t, (t - 1) * p.pat.r, st);
}

stencil_status read_device_error(int *flag)
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    int vs = 0, vw = 0, v3 = 0;
    stencil_status s = read_split_error(&vs);
    if (s != STENCIL_OK) return s;
    s = read_wide_error(&vw);
    if (s != STENCIL_OK) return s;
    s = read_wide3_error(&v3);
    if (s != STENCIL_OK) return s;
    *flag = v | vs | vw | v3;
    return STENCIL_OK;
}

}  // namespace gbs
