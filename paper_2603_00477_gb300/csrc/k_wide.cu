// k_wide.cu -- FP32 grids on the FP16 / BF16 tensor cores with wide MMAs
// (precisions f16, f16x3 and bf16x3): the Toeplitz (kernel-fusion) formulation of
// the paper's Sec. 2.2 with the roles of the two operands exchanged.
//
// On GB300 a tcgen05.mma of M = 128 costs a fixed ~90 cycles from one
// instruction to the next until its own arithmetic takes longer, so the
// useful work per instruction -- not the zero padding alone -- sets the rate
// of a Toeplitz kernel.  Here the Toeplitz factor of line a is the A operand
// (M = 128 output columns, K = the window of 128 + 2R input columns in
// blocks of 16) and the im2col of the input tile is the B operand (N = NR
// output rows, 256 where the operands fit): one instruction does
// 128 x 256 x 16 MACs, 16x those of the M = 128 x N = 32 form, in ~128
// cycles.
//
// The A operand needs no per-block copy.  With the output columns in reverse
// order (row m' of A is output column 127 - m'), A_a[m'][k] = w_a[k + m' - 127]
// depends on k + m' only, so the K-major core matrix (m' group g, k chunk c)
// of K block kb holds v_a[8 J + i + j] (row i, column j < 8) with
// J = 2 kb + c + g: one strip of 2 nkb + 15 core matrices per line serves
// every K block through a descriptor with LBO = SBO = 128 bytes.  A strip is
// zero outside core matrices 15 .. (127 + 2R) / 8, so the strips of
// consecutive lines overlap in their zeros (tc_wide_geom).
//
// The input tile (NR + 2R rows x 16 nkb columns, FP32) is read twice from
// global memory: once for its largest exponent, then again (from L2) to be
// scaled by a power of two and converted to FP16 or BF16 (hi, and lo = x - hi
// for the 3-product forms) in the chunk-column layout of k_tc.cu, where any 8 consecutive rows
// of a 16-byte chunk column form a K-major core matrix, so line a's B operand
// is a descriptor at row offset a.  The weights are scaled by a power of two
// likewise (hi and lo).  The scaled products accumulate in FP32 in TMEM
// (lane = output column, column = output row); the 3-product forms add
// hi*lo + lo*hi into the same accumulator.  The epilogue undoes both scalings exactly.
//
// Persistent, warp specialised, one CTA per SM (800 threads): warps 0-15 load
// and convert the next tile into the other operand buffer, one thread of
// warp 24 issues the MMAs into the other TMEM accumulator, warps 16-23 read
// the previous accumulator back (tcgen05.ld: one output column per thread,
// consecutive output rows in consecutive registers; two warps per TMEM lane
// quarter, each half of the rows) and store rows (32 consecutive columns per
// warp store).  Every wait is bounded.  Only
// interior points farther than (t-1) r from the boundary are written; the
// CUDA-core band kernel computes the others.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "launch.h"
#include "tc_layout.h"
#include "tc_ptx.cuh"

namespace gbs {

// Set when a bounded wait of this kernel runs out (each translation unit
// keeps its own error word; read_device_error reads them all).
__device__ int g_wide_error;

namespace wide {

using namespace tc;

constexpr int kMaxR = 12;
constexpr int kMaxLines = 2 * kMaxR + 1;
constexpr int TM = 128;         // output columns per tile (MMA M)
constexpr int KI = 16;          // K per instruction (kind::f16)
constexpr int kLoadWarps = 16;                // warps 0-15
constexpr int kLoaders = 32 * kLoadWarps;
constexpr int kEpiWarp = kLoadWarps;          // warps 16-23: TMEM lane quarter w % 4, half (w - 16) / 4
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kLoadWarps + kEpiWarps;  // warp 24
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kBatch = 8;                     // independent 16-byte loads in flight per loader thread
constexpr int kHeader = 1024;
constexpr unsigned long long kWaitCycles = 4ull << 30;       // ~2 s at 2 GHz
constexpr unsigned long long kDebugWaitCycles = 1ull << 22;  // ~2 ms: the test hook's limit

struct WideParams {
    double w[kMaxLines * kMaxLines];  // composite w^(t), (2R+1) x (2R+1), row-major
    unsigned char kb_lo[kMaxLines], kb_hi[kMaxLines];
    int R, rh, band, nkb, hs, delta, ew;
    int debug_unmet;  // test hook: wait once more on an mbarrier phase that never completes
    int vec16;        // 16-byte loads: stored rows are 16-byte multiples, tiles start aligned
    int xshift;       // tiles start xshift columns left of column 0
    int64_t Ey, Ex;
};

__device__ __forceinline__ float pow2f(int e)  // 2^e for -126 <= e <= 127
{
    return __int_as_float((e + 127) << 23);
}

// Operand type: FP16 (11 significant bits) or BF16 (8 significant bits, the
// range of FP32); packed conversions of two FP32 values and back.
template <bool BF>
struct Op;
template <>
struct Op<false> {
    using T2 = __half2;
    static constexpr uint32_t fmt = kFmtF16;
    __device__ static T2 pack(float a, float b) { return __floats2half2_rn(a, b); }
    __device__ static float2 unpack(T2 v) { return __half22float2(v); }
    __device__ static uint16_t bits(double w)
    {
        const __half h = __double2half(w);
        return *reinterpret_cast<const uint16_t *>(&h);
    }
    __device__ static double value(uint16_t b)
    {
        return (double)__half2float(*reinterpret_cast<const __half *>(&b));
    }
};
template <>
struct Op<true> {
    using T2 = __nv_bfloat162;
    static constexpr uint32_t fmt = kFmtBF16;
    __device__ static T2 pack(float a, float b) { return __floats2bfloat162_rn(a, b); }
    __device__ static float2 unpack(T2 v) { return __bfloat1622float2(v); }
    __device__ static uint16_t bits(double w)
    {
        const __nv_bfloat16 h = __double2bfloat16(w);
        return *reinterpret_cast<const uint16_t *>(&h);
    }
    __device__ static double value(uint16_t b)
    {
        return (double)__bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(&b));
    }
};

template <bool SPLIT, int NR, int NKB, bool BF, int NBUF>
__global__ void __launch_bounds__(kThreads, 1)
    tc2d_wide(const float *__restrict__ in, float *__restrict__ out, const __grid_constant__ WideParams p,
              int ntiles, int ntx)
{
    constexpr uint32_t kCols = 2 * NR;  // two accumulators of NR columns
    static_assert(kCols <= 512, "TMEM columns");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    int *abort_flag = reinterpret_cast<int *>(smem + 4);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 16);     // [2] operand buffer staged
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + 32);     // [2] MMAs of a tile complete
    uint64_t *accfree = reinterpret_cast<uint64_t *>(smem + 48);  // [2] accumulator drained
    uint64_t *maxb = reinterpret_cast<uint64_t *>(smem + 64);     // [2] exponent exchange
    uint64_t *eub = reinterpret_cast<uint64_t *>(smem + 80);      // [4] a tile's scale published
    int *wmax = reinterpret_cast<int *>(smem + 128);              // [2][kLoadWarps]
    int *eus = reinterpret_cast<int *>(smem + 256);               // [4] input scale exponent per tile
    constexpr int nkb = NKB;
    const int R = p.R, HS = p.hs, lines = 2 * R + 1;
    const uint32_t strip_bytes = (uint32_t)(2 * R * p.delta + 2 * nkb + 15) * 128;
    const uint32_t in_bytes = (uint32_t)(2 * nkb) * HS * 16;
    unsigned char *Whi = smem + kHeader;
    unsigned char *Wlo = Whi + strip_bytes;
    unsigned char *ibase = Whi + strip_bytes * (SPLIT ? 2 : 1);
    // operand buffer b (b = 0 when NBUF = 1): hi at ibase + b in_bytes, lo
    // (the 3-product forms) NBUF in_bytes further
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t Ey = p.Ey, Ex = p.Ex, rh = p.rh;
    const int64_t ny = Ey - 2 * rh, nx = Ex - 2 * rh;

    if (warp == kMmaWarp) tmem_alloc(tmem_slot, kCols);
    if (tid == 0) {
        *abort_flag = 0;
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], kLoaders);
            mbar_init(&done[b], 1);
            mbar_init(&accfree[b], 32 * kEpiWarps);
            mbar_init(&maxb[b], kLoaders);
        }
        for (int s = 0; s < 4; ++s) mbar_init(&eub[s], 1);
        fence_mbar_init();
    }
    // weight strips: zero them, then write the non-zero core matrices
    const uint32_t wbytes = strip_bytes * (SPLIT ? 2 : 1);
    for (uint32_t i = (uint32_t)tid * 16; i < wbytes; i += kThreads * 16)
        *reinterpret_cast<uint4 *>(Whi + i) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    {
        const int jlo = 15, jn = (127 + 2 * R) / 8 - jlo + 1;
        const double wsc = ldexp(1.0, 15 - p.ew);  // |w| 2^(15 - ew) < 2^15: exact scaling
        for (int e = tid; e < lines * jn * 64; e += kThreads) {
            const int ii = (e >> 3) & 7, jj = e & 7, rest = e >> 6;
            const int J = jlo + rest % jn, ai = rest / jn;
            const int idx = 8 * J + ii + jj - 127;  // tap offset + R of output column 127 - (8g + ii)
            if (idx < 0 || idx > 2 * R) continue;
            const double wv = p.w[ai * lines + idx] * wsc;
            const uint32_t off = (uint32_t)(ai * p.delta + J) * 128 + ii * 16 + jj * 2;
            const uint16_t h = Op<BF>::bits(wv);
            *reinterpret_cast<uint16_t *>(Whi + off) = h;
            if (SPLIT) *reinterpret_cast<uint16_t *>(Wlo + off) = Op<BF>::bits(wv - Op<BF>::value(h));
        }
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
        *Y0 = rh + (int64_t)(id / ntx) * NR;
        *X0 = (int64_t)(id % ntx) * TM - p.xshift;
    };

    if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(Op<BF>::fmt, TM, NR);
            const uint64_t a0 = smem_desc(smem_u32(Whi), 128, 128);
            const uint64_t dlo_a = (uint64_t)(strip_bytes >> 4);
            int k = 0;
            for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
                const int b = k & 1;
                if (!bounded_wait(&full[b], (k >> 1) & 1, kWaitCycles)) break;
                if (k >= 2 && !bounded_wait(&accfree[b], ((k - 2) >> 1) & 1, kWaitCycles)) break;
                fence_after_thread_sync();
                const uint64_t b0 = smem_desc(smem_u32(ibase + (NBUF == 2 ? b : 0) * in_bytes), (uint32_t)HS * 16, 128);
                const uint64_t dlo_b = (uint64_t)((NBUF * in_bytes) >> 4);
                const uint32_t d = tmem + (uint32_t)(b * NR);
                uint32_t acc = 0;
                for (int ai = 0; ai < lines; ++ai) {
                    const int klo = p.kb_lo[ai], khi = p.kb_hi[ai];
                    // strip of line ai from K block klo (two core matrices per block);
                    // input rows from row ai, chunk columns from 2 klo
                    uint64_t da = a0 + (uint64_t)(ai * p.delta + 2 * klo) * 8;
                    uint64_t db = b0 + (uint64_t)(2 * klo) * HS + (uint64_t)ai;
                    for (int kb = klo; kb <= khi; ++kb) {
                        mma_f16(d, da, db, idesc, acc);
                        if (SPLIT) {
                            mma_f16(d, da, db + dlo_b, idesc, 1);
                            mma_f16(d, da + dlo_a, db, idesc, 1);
                        }
                        acc = 1;
                        da += 16;
                        db += (uint64_t)(2 * HS);
                    }
                }
                mma_commit(&done[b]);
            }
            // the last tiles' MMAs complete before the TMEM is released
            for (int j = k - 2; j < k; ++j)
                if (j >= 0) {
                    const unsigned long long t0 = clock64();
                    while (!mbar_try_wait(&done[j & 1], (j >> 1) & 1) && clock64() - t0 < kWaitCycles) {
                    }
                }
        }
        __syncwarp();
    } else if (warp < kEpiWarp) {
        // ---------------- loaders / converters ----------------
        constexpr int F4 = 4 * NKB;  // float4 per staged row (16 NKB columns)
        const int rows = NR + 2 * R, items = rows * F4;
        const bool vec16 = p.vec16 != 0;
        auto ld4 = [&](int64_t Y0, int64_t X0, int row, int c4) -> float4 {
            const int64_t gy = Y0 - R + row, gx = X0 - R + 4 * c4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy < 0 || gy >= Ey) return v;
            const float *g = in + gy * Ex;
            if (vec16) {
                // X0 - R is a multiple of 4: the 4 values lie wholly inside or outside the row
                if (gx >= 0 && gx < Ex) v = __ldcg(reinterpret_cast<const float4 *>(g + gx));
                return v;
            }
            if (gx >= 0 && gx < Ex) v.x = __ldcg(g + gx);
            if (gx + 1 >= 0 && gx + 1 < Ex) v.y = __ldcg(g + gx + 1);
            if (gx + 2 >= 0 && gx + 2 < Ex) v.z = __ldcg(g + gx + 2);
            if (gx + 3 >= 0 && gx + 3 < Ex) v.w = __ldcg(g + gx + 3);
            return v;
        };
        // ask L2 for tile `id`'s input rows (one prefetch per 128 bytes, every
        // address inside the stored array), so that both passes over it wait
        // on L2 rather than DRAM latency
        auto prefetch_l2 = [&](int id) {
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            const int64_t gx_lo = max((int64_t)0, X0 - R), gx_hi = min(Ex, X0 - R + 16 * NKB);
            if (gx_lo >= gx_hi) return;
            const int lines = (int)((gx_hi - gx_lo + 31) / 32);
            for (int e = tid; e < rows * lines; e += kLoaders) {
                const int row = e / lines, l = e - (e / lines) * lines;
                const int64_t gy = Y0 - R + row;
                if (gy < 0 || gy >= Ey) continue;
                const int64_t gx = min(gx_lo + 32 * (int64_t)l, gx_hi - 1);
                asm volatile("prefetch.global.L2 [%0];" ::"l"(in + gy * Ex + gx));
            }
        };
        int k = 0;
        for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
            const int b = k & 1;
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            if (id + (int)gridDim.x < ntiles) prefetch_l2(id + gridDim.x);
            // Interior tiles (the staged region inside the stored array, 16-byte
            // rows): no per-load bounds tests; thread tid takes the float4 items
            // i = tid + m kLoaders, whose (row, column) advance by a constant step.
            const bool fast = vec16 && Y0 - R >= 0 && Y0 - R + rows <= Ey && X0 - R >= 0 &&
                              X0 - R + 16 * NKB <= Ex;
            const float *g0 = in + (Y0 - R) * Ex + (X0 - R);
            constexpr int step_r = kLoaders / F4, step_c = kLoaders % F4;
            auto load = [&](int i, int r, int c) -> float4 {
                return fast ? __ldcg(reinterpret_cast<const float4 *>(g0 + (int64_t)r * Ex + 4 * c))
                            : ld4(Y0, X0, i / F4, i % F4);
            };
            // pass 1: the tile's largest |x| as an unsigned integer (IEEE order), then its exponent
            unsigned mxu = 0;
            {
                int row = tid / F4, c4 = tid % F4;
                for (int i0 = tid; i0 < items; i0 += kBatch * kLoaders) {
                    float4 v[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + u * kLoaders;
                        v[u] = i < items ? load(i, row, c4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        row += step_r;
                        c4 += step_c;
                        if (c4 >= F4) {
                            c4 -= F4;
                            ++row;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u)
                        mxu = max(mxu, max(max(__float_as_uint(v[u].x) & 0x7fffffffu, __float_as_uint(v[u].y) & 0x7fffffffu),
                                           max(__float_as_uint(v[u].z) & 0x7fffffffu, __float_as_uint(v[u].w) & 0x7fffffffu)));
                }
            }
            const int mx = (int)(__reduce_max_sync(0xffffffffu, mxu) >> 23);
            if (lane == 0) wmax[b * kLoadWarps + warp] = mx;
            __syncwarp();
            mbar_arrive(&maxb[b]);
            if (!bounded_wait(&maxb[b], (k >> 1) & 1, kWaitCycles)) break;
            int emax = wmax[b * kLoadWarps];
#pragma unroll
            for (int w = 1; w < kLoadWarps; ++w) emax = max(emax, wmax[b * kLoadWarps + w]);
            // |x| < 2^(emax - 126): x 2^es < 2^15 with es = 141 - emax (clamped)
            const int es = max(-126, min(127, 141 - emax));
            const float xs = pow2f(es);
            // the operand buffer is free once the MMAs of tile k - NBUF completed
            if (NBUF == 2 && k >= 2 && !bounded_wait(&done[b], ((k - 2) >> 1) & 1, kWaitCycles)) break;
            if (NBUF == 1 && k >= 1 && !bounded_wait(&done[b ^ 1], ((k - 1) >> 1) & 1, kWaitCycles)) break;
            // publish the scale: slot k & 3 was last read by the epilogue of tile
            // k - 4, which finished before the MMAs of tile k - 2 could start
            // (and those precede the MMAs of tile k - NBUF waited for above)
            if (tid == 0) {
                eus[k & 3] = es;
                mbar_arrive(&eub[k & 3]);
            }
            // pass 2: scale, convert, store 4 FP16/BF16 values (8 bytes) per float4
            {
                unsigned char *hi = ibase + (NBUF == 2 ? b : 0) * in_bytes, *lo = hi + NBUF * in_bytes;
                int row = tid / F4, c4 = tid % F4;
                for (int i0 = tid; i0 < items; i0 += kBatch * kLoaders) {
                    float4 vb[kBatch];
                    int rr[kBatch], cc[kBatch];
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        const int i = i0 + u * kLoaders;
                        rr[u] = row;
                        cc[u] = c4;
                        vb[u] = i < items ? load(i, row, c4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        row += step_r;
                        c4 += step_c;
                        if (c4 >= F4) {
                            c4 -= F4;
                            ++row;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kBatch; ++u) {
                        if (i0 + u * kLoaders >= items) break;
                        const float4 v = vb[u];
                        const float x0 = v.x * xs, x1 = v.y * xs, x2 = v.z * xs, x3 = v.w * xs;
                        const typename Op<BF>::T2 h01 = Op<BF>::pack(x0, x1), h23 = Op<BF>::pack(x2, x3);
                        const uint32_t off = (uint32_t)((cc[u] >> 1) * HS + rr[u]) * 16 + (uint32_t)(cc[u] & 1) * 8;
                        uint2 hv;
                        hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                        hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                        *reinterpret_cast<uint2 *>(hi + off) = hv;
                        if (SPLIT) {
                            const float2 f01 = Op<BF>::unpack(h01), f23 = Op<BF>::unpack(h23);
                            const typename Op<BF>::T2 l01 = Op<BF>::pack(x0 - f01.x, x1 - f01.y);
                            const typename Op<BF>::T2 l23 = Op<BF>::pack(x2 - f23.x, x3 - f23.y);
                            uint2 lv;
                            lv.x = *reinterpret_cast<const uint32_t *>(&l01);
                            lv.y = *reinterpret_cast<const uint32_t *>(&l23);
                            *reinterpret_cast<uint2 *>(lo + off) = lv;
                        }
                    }
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&full[b]);
        }
    } else {
        // ---------------- epilogue (warps 16-23) ----------------
        // warp w reads TMEM lanes 32 q .. 32 q + 31 (q = w % 4, the lane quarter
        // a warp may access) for the accumulator columns (output rows) of half h
        const int q = (warp - kEpiWarp) & 3, h = (warp - kEpiWarp) >> 2;
        const int m = TM - 1 - (32 * q + lane);
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
        int k = 0;
        bool ok = true;
        for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
            const int b = k & 1;
            if (!bounded_wait(&eub[k & 3], (k >> 2) & 1, kWaitCycles)) {
                ok = false;
                break;
            }
            const int es = eus[k & 3];
            if (!bounded_wait(&done[b], (k >> 1) & 1, kWaitCycles)) {
                ok = false;
                break;
            }
            fence_after_thread_sync();
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            const int64_t gx = X0 + m, ix = gx - rh;
            const bool colok = ix >= p.band && ix < nx - p.band;
            // rows n of the tile written: interior rows iy = Y0 - rh + n in [band, ny - band)
            const int n_lo = (int)max((int64_t)0, p.band - (Y0 - rh));
            const int n_hi = (int)min((int64_t)NR, ny - p.band - (Y0 - rh));
            // out = acc 2^(ew - 15 - es), as two in-range powers of two
            const int e = p.ew - 15 - es, e1 = e / 2, e2 = e - e1;
            const float s1 = pow2f(max(-126, min(127, e1))), s2 = pow2f(max(-126, min(127, e2)));
            float *o = out + Y0 * Ex + gx;
            for (int n0 = h * (NR / 2); n0 < (h + 1) * (NR / 2); n0 += 16) {
                uint32_t v[16];
                __syncwarp();
                tmem_ld_32x32b_x16(lane_base + (uint32_t)(b * NR + n0), v);
                tmem_ld_wait();
                if (n0 >= n_hi) break;  // rows below the written band
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + j;
                    if (colok && n >= n_lo && n < n_hi) o[(int64_t)n * Ex] = __uint_as_float(v[j]) * s1 * s2;
                }
            }
            fence_before_thread_sync();
            mbar_arrive(&accfree[b]);
        }
        if (ok && p.debug_unmet && k > 0) {
            // test hook: a phase that never completes -> the bounded wait reports it
            bounded_wait(&done[(k - 1) & 1], (((k - 1) >> 1) & 1) ^ 1, kDebugWaitCycles);
        }
    }
    fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *(volatile int *)abort_flag) atomicExch(&g_wide_error, 1);
    if (warp == kMmaWarp) tmem_dealloc(tmem, kCols);
}

}  // namespace wide

namespace {

template <bool SPLIT, int NR, int NKB, bool BF, int NBUF>
stencil_status launch_wide_n(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    using namespace wide;
    const int r = p.pat.r, R = t * r;
    if (R > kMaxR) return fail(STENCIL_ERR_UNSUPPORTED, "wide FP16 path: fused radius t*r must be <= 12");
    const WideGeom g = tc_wide_geom(R, NR, SPLIT, NBUF);
    if (g.smem > 227 * 1024) return fail(STENCIL_ERR_UNSUPPORTED, "wide FP16 tile does not fit in shared memory");
    if (g.nkb != NKB) return fail(STENCIL_ERR_INTERNAL, "wide FP16 path: K blocks");
    const TcLines L = tc_lines_2d(p.pat.shape, r, t, TM, KI);
    if (L.nkb != g.nkb) return fail(STENCIL_ERR_INTERNAL, "wide FP16 path: K blocks");
    WideParams wp;
    std::memset(&wp, 0, sizeof(wp));
    const std::vector<double> wt = compose_dense(p.pat, p.w, t);
    const int lines = 2 * R + 1;
    double wmax = 0;
    for (int i = 0; i < lines * lines; i++) {
        wp.w[i] = wt[i];
        wmax = std::max(wmax, std::fabs(wt[i]));
    }
    for (int a = 0; a < lines; a++) {
        wp.kb_lo[a] = (unsigned char)L.kb_lo[a];
        wp.kb_hi[a] = (unsigned char)L.kb_hi[a];
        if (L.kb_lo[a] > L.kb_hi[a]) {  // empty line
            wp.kb_lo[a] = 1;
            wp.kb_hi[a] = 0;
        }
    }
    wp.R = R;
    wp.rh = r;
    wp.band = (t - 1) * r;
    wp.nkb = g.nkb;
    wp.hs = g.hs;
    wp.delta = g.delta;
    wp.ew = 0;
    if (wmax > 0) std::frexp(wmax, &wp.ew);  // wmax < 2^ew
    wp.debug_unmet = p.debug_unmet_wait;
    wp.Ey = p.ext[1];
    wp.Ex = p.ext[2];
    wp.vec16 = (p.ext[2] % 4 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
    wp.xshift = wp.vec16 ? (4 - R % 4) % 4 : 0;  // (tile start - R) a multiple of 4
    auto kern = tc2d_wide<SPLIT, NR, NKB, BF, NBUF>;
    stencil_status s = ensure_smem((const void *)kern, g.smem);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t nty = (p.dims[1] + NR - 1) / NR, ntx = (p.ext[2] + wp.xshift + TM - 1) / TM;
    const int64_t ntiles = nty * ntx;
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
    kern<<<grid, kThreads, g.smem, st>>>((const float *)in, (float *)out, wp, (int)ntiles, (int)ntx);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "tc2d_wide launch");
}

}  // namespace

stencil_status launch_wide_sweep(const Plan &p, const void *in, void *out, int t, bool split, bool bf16,
                                 cudaStream_t st)
{
    const WideTile wt = tc_wide_tile(p.pat.r, t, split);
    const int nr = wt.nr, nb = wt.nbuf;
    const int nkb = tc_wide_geom(t * p.pat.r, 128, split).nkb;  // 9 (R <= 8) or 10
    // the (N, K blocks, buffers) triples tc_wide_tile can pick
    if (split) {
#define GBS_WIDE_SPLIT(BFV)                                                                                   \
    if (nr == 128 && nkb == 9 && nb == 2) return launch_wide_n<true, 128, 9, BFV, 2>(p, in, out, t, st);     \
    if (nr == 128 && nkb == 9 && nb == 1) return launch_wide_n<true, 128, 9, BFV, 1>(p, in, out, t, st);     \
    if (nr == 128 && nkb == 10 && nb == 1) return launch_wide_n<true, 128, 10, BFV, 1>(p, in, out, t, st);
        if (bf16) {
            GBS_WIDE_SPLIT(true)
        } else {
            GBS_WIDE_SPLIT(false)
        }
#undef GBS_WIDE_SPLIT
    } else if (!bf16) {
        if (nr == 256 && nkb == 9 && nb == 2) return launch_wide_n<false, 256, 9, false, 2>(p, in, out, t, st);
        if (nr == 256 && nkb == 10 && nb == 2) return launch_wide_n<false, 256, 10, false, 2>(p, in, out, t, st);
        if (nr == 128 && nkb == 10 && nb == 2) return launch_wide_n<false, 128, 10, false, 2>(p, in, out, t, st);
    }
    return fail(STENCIL_ERR_UNSUPPORTED, "wide FP16 tile does not fit in shared memory");
}

stencil_status read_wide_error(int *flag)
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_wide_error, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_wide_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the wide kernel's error word");
    *flag = v;
    return STENCIL_OK;
}

}  // namespace gbs
