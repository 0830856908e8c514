// k_split.cu -- FP64 stencil sweeps on the FP16 tensor cores by exact
// splitting (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), applied
// to the Toeplitz (kernel-fusion) formulation of the paper's Sec. 2.2.
//
// GB300 runs FP64 at 1.26 TFLOP/s on both the FMA pipe and the FP64 MMA, so
// the paper's Eq. 19 (alpha < S P_TC / P_CU) never holds for FP64 operands.
// The FP16 tensor core is ~1800x faster; this kernel moves the FP64 work there
// without losing FP64 accuracy:
//
//   * every staged input tile is written in fixed point relative to its
//     largest exponent E_u: V = round(u * 2^(NB - E_u)), |V| <= 2^NB
//     (NB = S*b - 1 >= 53 bits), and V is cut into S balanced b-bit digits
//     a_0..a_{S-1} (V = sum_i a_i 2^(b(S-1-i)), |a_i| <= 2^(b-1)), each an
//     exact FP16 integer;
//   * the composite weights w^(t) are cut the same way on the host (digits
//     b_j, exponent E_w);
//   * one tcgen05.mma kind::f16 per A slice i multiplies the im2col window of
//     a_i by [T(b_0) | T(b_1) | ... | T(b_{S-1-i})] (the Toeplitz blocks of the
//     weight digits side by side along N), accumulating the product of slice
//     pair (i, j) into the FP32 accumulator of its level L = i + j in TMEM;
//     products of |a_i b_j| <= 2^(2b-2) are exact and the host checks that
//     every level's sum of absolute values stays below 2^24 (choosing b = 9
//     or 8), so every accumulator holds its exact integer sum S_L
//     whatever the order and rounding of the tensor core's additions;
//   * the epilogue converts S_L to integers, combines
//     T = sum_L S_L 2^(b(S-1-L) - D) in 64-bit integers (D drops the bits
//     below ~2^-55 of the largest term) and scales T by
//     2^(b(S-1) + D + E_u + E_w - 2 NB).  Levels L >= S (below 2^-bS of the
//     leading term) are not formed.
//
// Per fused sweep the result is the exact stencil sum of the digit
// representations (53 significant bits of u relative to the tile's maximum,
// 53 of w^(t)), rounded once: the error is a few units of 2^-53 of
// max|u| * sum|w| per sweep (normwise), like FP64 arithmetic.
//
// The kernel is warp specialised and persistent (one CTA per SM, 544
// threads): warp 16 issues the MMAs; warps 0-15 load the next tile's FP64
// input into registers, reduce its exponent, cut it into digit slices in
// shared memory (chunk-column K-major layout, the implicit im2col of k_tc.cu)
// and drain the previous tile's accumulators (double-buffered TMEM).  Only
// interior points farther than (t-1) r from the boundary are written; the
// CUDA-core band kernel computes the others.
#include <cuda_fp16.h>

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

// Set when a bounded wait of this kernel runs out (the library is built
// without relocatable device code, so each translation unit keeps its own
// error word; read_device_error reads them all).
__device__ int g_split_error;

namespace split {

using namespace tc;

constexpr int kMaxR = 8;                       // N = 16, K window <= 32: two K blocks per line
constexpr int kMaxLines = 2 * kMaxR + 1;
constexpr int kMaxS = 7;  // S = 8 (7-bit digits) is only needed at fused radii whose tiles do not fit
constexpr int TM = 128, TN = 16, KI = 16;      // MMA M, N per accumulator block, K per instruction
constexpr int kNkb = 2;                        // K blocks per line (window 16 + 2R <= 32)
constexpr int kWorkerWarps = 16;
constexpr int kWorkers = 32 * kWorkerWarps;    // warps 0-15; warp 16 issues the MMAs
constexpr int kThreads = kWorkers + 32;
constexpr int kItemsPerThread = 2;             // (TM + 2R) * NCH <= 144 * 6 = 864 <= 2 * 512
constexpr int kHeader = 256;                   // TMEM slot, abort word, mbarriers, exponent slots

struct SplitParams {
    short wd[kMaxS][kMaxLines * kMaxLines];  // weight digits b_j of w^(t), (2R+1)^2 row-major
    unsigned char kb_lo[kMaxLines], kb_hi[kMaxLines];
    int R, rh, band, hs, nch;
    int scale0;        // b(S-1) + D + E_w - 2 NB - 1022: the result scale is 2^(scale0 + emax)
    int vec16;         // rows start on 16-byte boundaries and X0 - R is even: 16-byte loads
    int debug_unmet;   // test hook: a wait on an mbarrier phase that never completes
    int64_t Ey, Ex;
};

template <int S>
struct Digits {
    static constexpr int b = S == 6 ? 9 : (S == 7 ? 8 : 7);
    static constexpr int NB = S * b - 1;                        // fixed-point bits of |V|
    static constexpr int D = (24 + b * (S - 1) - 62) > 0 ? (24 + b * (S - 1) - 62) : 0;
};

constexpr unsigned long long kWaitCycles = 4ull << 30;         // ~2 s at 2 GHz
constexpr unsigned long long kDebugWaitCycles = 1ull << 22;    // ~2 ms: the test hook's limit

__device__ __forceinline__ bool wait_cycles(uint64_t *mbar, uint32_t phase, unsigned long long limit)
{
    const unsigned long long t0 = clock64();
    while (!mbar_try_wait(mbar, phase)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// Fixed-point value of x relative to the tile exponent emax (the largest
// biased exponent of the tile, >= 1): V = round(x * 2^(NB - E_u)),
// E_u = emax - 1022, computed from the bits of x with integer operations.
template <int S>
__device__ __forceinline__ long long fixed_point(unsigned long long X, int emax)
{
    constexpr int NB = Digits<S>::NB;
    int ex = (int)((X >> 52) & 0x7FF);
    unsigned long long m = X & ((1ull << 52) - 1);
    if (ex) m |= 1ull << 52;
    else ex = 1;
    const int sh = (53 - NB) + (emax - ex);
    unsigned long long v;
    if (sh <= 0) v = m << (-sh);
    else if (sh < 62) v = (m + (1ull << (sh - 1))) >> sh;
    else v = 0;
    const long long V = (long long)v;
    return (X >> 63) ? -V : V;
}

// The S balanced b-bit digits of V (top first), each as the FP16 bit pattern
// of 1536 + digit (exact: 1536 +- 2^(b-1) lies in [1024, 2048), where FP16
// steps by 1); 1536 is subtracted after packing two digits into a half2.
// V is split at 3b bits into a non-negative low word (three digits, then a
// carry of 0 or 1) and a signed high word (the rest), so every step is a
// 32-bit operation: |V| <= 2^(S b - 1) leaves |V >> 3b| < 2^31.
template <int S>
__device__ __forceinline__ void digits16(long long V, unsigned short (&h)[S])
{
    constexpr int b = Digits<S>::b;
    constexpr int half = 1 << (b - 1), mask = (1 << b) - 1;
    constexpr int LO = 3;  // digits in the low word
    int lo = (int)((unsigned long long)V & ((1ull << (LO * b)) - 1));
    int hi = (int)(V >> (LO * b));
#pragma unroll
    for (int i = S - 1; i >= S - LO; --i) {
        const int d = ((lo & mask) ^ half) - half;  // in [-2^(b-1), 2^(b-1))
        h[i] = (unsigned short)(0x6600 + d);
        lo = (lo - d) >> b;
    }
    hi += lo;  // the carry out of the low word
#pragma unroll
    for (int i = S - LO - 1; i >= 1; --i) {
        const int d = ((hi & mask) ^ half) - half;
        h[i] = (unsigned short)(0x6600 + d);
        hi = (hi - d) >> b;
    }
    h[0] = (unsigned short)(0x6600 + hi);  // |top digit| <= 2^(b-1)
}

__device__ __forceinline__ uint32_t hsub1536(uint32_t packed)
{
    const __half2 v = *reinterpret_cast<const __half2 *>(&packed);
    const __half2 r = __hsub2(v, __half2half2(__ushort_as_half((unsigned short)0x6600)));
    return *reinterpret_cast<const uint32_t *>(&r);
}

template <int S, int NACC>
__global__ void __launch_bounds__(kThreads, 1)
    tc2d_split(const double *__restrict__ in, double *__restrict__ out, const __grid_constant__ SplitParams p,
               int ntiles, int ntx)
{
    constexpr int b = Digits<S>::b, D = Digits<S>::D;
    constexpr int TX = NACC * TN;
    constexpr uint32_t kSet = (uint32_t)TN * S * NACC;  // TMEM columns of one accumulator set
    constexpr uint32_t kCols = 2 * kSet <= 256 ? 256 : 512;
    constexpr uint32_t kBlk = 2u * S * 256u;             // bytes of one B block: 16 S rows (n) x 16 k
    static_assert(2 * kSet <= 512, "two accumulator sets must fit in TMEM");

    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    int *abort_flag = reinterpret_cast<int *>(smem + 4);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 16);   // [2]
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + 32);   // [2]
    uint64_t *freeb = reinterpret_cast<uint64_t *>(smem + 48);  // [2]
    uint64_t *emaxb = reinterpret_cast<uint64_t *>(smem + 64);  // [2]: the tile exponent is reduced
    int *wmax = reinterpret_cast<int *>(smem + 80);             // [2][kWorkerWarps], bytes 80..207
    static_assert(80 + 2 * kWorkerWarps * sizeof(int) <= kHeader, "the header holds the barriers and exponents");
    const int R = p.R, HS = p.hs, NCH = p.nch;
    const int lines = 2 * R + 1;
    const uint32_t slice_bytes = (uint32_t)NCH * HS * 16;
    const uint32_t a_bytes = slice_bytes * S;
    unsigned char *Bm = smem + kHeader;
    unsigned char *A[2] = {Bm + (size_t)lines * kNkb * kBlk, Bm + (size_t)lines * kNkb * kBlk + a_bytes};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t Ey = p.Ey, Ex = p.Ex, rh = p.rh;
    const int64_t ny = Ey - 2 * rh, nx = Ex - 2 * rh;

    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    if (tid == 0) {
        *abort_flag = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], kWorkers);
            mbar_init(&done[i], 1);
            mbar_init(&freeb[i], kWorkers);
            mbar_init(&emaxb[i], kWorkers);
        }
        fence_mbar_init();
    }
    // Toeplitz blocks of the weight digits: block (line a, kb) holds, for
    // j = 0..S-1, rows n' = 16 j + n (output column n) and k = 0..15 of the
    // window, B[n'][k] = b_j(a, kb*16 + k - n - R) in its band; K-major core
    // matrices (n-group g, k-chunk c) at g*256 + c*128.
    const int bent = lines * kNkb * TN * S * KI;
    for (int idx = tid; idx < bent; idx += blockDim.x) {
        const int k = idx % KI, nn = (idx / KI) % (TN * S), blk = idx / (KI * TN * S);
        const int a = blk / kNkb, kb = blk % kNkb;
        const int j = nn / TN, n = nn % TN;
        const int c = kb * KI + k - n - R;
        const int dgt = (c >= -R && c <= R) ? p.wd[j][a * lines + (c + R)] : 0;
        const uint32_t off = blk * kBlk + (nn / 8) * 256 + (k / 8) * 128 + (nn % 8) * 16 + (k % 8) * 2;
        *reinterpret_cast<__half *>(Bm + off) = __int2half_rn(dgt);
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
        *X0 = rh + (int64_t)(id % ntx) * TX;
    };

    if (warp == kWorkerWarps) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t lbo_a = (uint32_t)HS * 16;
            const uint64_t db0 = smem_desc(smem_u32(Bm), 128, 256);
            int k = 0;
            for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
                const int bf = k & 1;
                if (!bounded_wait(&full[bf], (k >> 1) & 1, kWaitCycles)) break;
                if (k >= 2 && !bounded_wait(&freeb[bf], ((k - 2) >> 1) & 1, kWaitCycles)) break;
                fence_after_thread_sync();
                const uint64_t da0 = smem_desc(smem_u32(A[bf]), lbo_a, 128);
                const uint32_t dset = tmem + bf * kSet;
                uint32_t first = 1;
                for (int a = 0; a < lines; ++a) {
                    for (int kb = p.kb_lo[a]; kb <= p.kb_hi[a]; ++kb) {
                        const uint64_t db = db0 + (uint64_t)((uint32_t)(a * kNkb + kb) * kBlk >> 4);
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const uint32_t idesc = instr_desc(kFmtF16, TM, TN * (S - i));
#pragma unroll
                            for (int q = 0; q < NACC; ++q) {
                                // A slice i, window of column block q, K block kb, line a
                                const uint32_t aoff = i * slice_bytes + (uint32_t)((2 * q + 2 * kb) * HS + a) * 16;
                                mma_f16(dset + (uint32_t)(q * TN * S + TN * i), da0 + (aoff >> 4), db, idesc,
                                        (first && i == 0) ? 0u : 1u);
                            }
                        }
                        first = 0;
                    }
                }
                mma_commit(&done[bf]);
            }
            // the last MMAs finish before TMEM can be freed
            if (k >= 1) wait_cycles(&done[(k - 1) & 1], ((k - 1) >> 1) & 1, kWaitCycles);
            if (k >= 2) wait_cycles(&done[(k - 2) & 1], ((k - 2) >> 1) & 1, kWaitCycles);
        }
        __syncwarp();
    } else {
        // -------- loaders / digit cutters and epilogue (warps 0-15) --------
        const int rows = TM + 2 * R;
        const int nitems = rows * NCH;
        double v[kItemsPerThread][8];
        auto prefetch = [&](int id) {
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
#pragma unroll
            for (int j = 0; j < kItemsPerThread; ++j) {
                const int it = tid + kWorkers * j;
                const int c = it / rows, row = it - (it / rows) * rows;
                const int64_t gy = Y0 - R + row, gx0 = X0 - R + 8 * c;
                const bool rowok = it < nitems && gy >= 0 && gy < Ey;
                const double *src = in + (rowok ? gy : 0) * Ex;
                if (p.vec16 && rowok && gx0 >= 0 && gx0 + 8 <= Ex) {
                    // the eight values lie in the row and start on a 16-byte boundary
                    const double2 *s2 = reinterpret_cast<const double2 *>(src + gx0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const double2 d2 = __ldg(s2 + e);
                        v[j][2 * e] = d2.x;
                        v[j][2 * e + 1] = d2.y;
                    }
                    continue;
                }
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int64_t gx = gx0 + e;
                    v[j][e] = (rowok && gx >= 0 && gx < Ex) ? __ldg(src + gx) : 0.0;
                }
            }
        };
        // largest biased exponent of the staged tile k (>= 1) over the
        // workers: per-warp maxima in shared memory, exchanged through an
        // mbarrier with a bounded wait (-1: the wait gave up)
        auto tile_emax = [&](int k) -> int {
            const int slot = k & 1;
            int mx = 1;
#pragma unroll
            for (int j = 0; j < kItemsPerThread; ++j)
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    mx = max(mx, (int)((__double_as_longlong(v[j][e]) >> 52) & 0x7FF));
            mx = __reduce_max_sync(0xffffffffu, (unsigned)mx);
            if (lane == 0) wmax[slot * kWorkerWarps + warp] = mx;
            __syncwarp();
            mbar_arrive(&emaxb[slot]);
            if (!bounded_wait(&emaxb[slot], (k >> 1) & 1, kWaitCycles)) return -1;
            int m = wmax[slot * kWorkerWarps];
#pragma unroll
            for (int w = 1; w < kWorkerWarps; ++w) m = max(m, wmax[slot * kWorkerWarps + w]);
            return m;
        };
        auto cut = [&](unsigned char *Abuf, int emax) {
#pragma unroll
            for (int j = 0; j < kItemsPerThread; ++j) {
                const int it = tid + kWorkers * j;
                if (it >= nitems) continue;
                const int c = it / rows, row = it - (it / rows) * rows;
                uint32_t pk[S][4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    unsigned short h0[S], h1[S];
                    digits16<S>(fixed_point<S>((unsigned long long)__double_as_longlong(v[j][e]), emax), h0);
                    digits16<S>(fixed_point<S>((unsigned long long)__double_as_longlong(v[j][e + 1]), emax), h1);
#pragma unroll
                    for (int i = 0; i < S; ++i) pk[i][e / 2] = hsub1536((uint32_t)h0[i] | ((uint32_t)h1[i] << 16));
                }
                const uint32_t off = (uint32_t)(c * HS + row) * 16;
#pragma unroll
                for (int i = 0; i < S; ++i)
                    *reinterpret_cast<uint4 *>(Abuf + i * slice_bytes + off) =
                        make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
            }
        };
        // accumulators of tile `id` (set `bf`, tile exponent emax) -> out
        auto epilogue = [&](int id, int bf, int emax) {
            int64_t Y0, X0;
            origin(id, &Y0, &X0);
            const int m = (warp & 3) * 32 + lane;
            const int64_t gy = Y0 + m, iy = gy - rh;
            const bool rowok = iy < ny && iy >= p.band && ny - 1 - iy >= p.band;
            const uint32_t lane_base = tmem + bf * kSet + ((uint32_t)((warp & 3) * 32) << 16);
            const bool nan_tile = emax == 0x7FF;
            // the result is T * 2^sc.  (double)T has a biased exponent in
            // [1023, 1085] (1 <= |T| < 2^63), so adding sc to the exponent
            // field scales exactly when that stays a normal number; otherwise
            // two multiplications by powers of two do it
            const int sc = p.scale0 + emax;
            const bool exp_add = sc >= 1 - 1023 && sc <= 2046 - 1085;
            const int sc1 = sc / 2, sc2 = sc - sc1;
            const double s1 = __longlong_as_double((long long)(max(-1022, min(1023, sc1)) + 1023) << 52);
            const double s2 = __longlong_as_double((long long)(max(-1022, min(1023, sc2)) + 1023) << 52);
            const long long sc_bits = (long long)sc << 52;
            for (int g = warp >> 2; g < 2 * NACC; g += kWorkerWarps / 4) {
                const int q = g >> 1, h = g & 1;
                // T = sum_L S_L 2^(b(S-1-L) - D), one level at a time
                long long T[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) T[c] = 0;
#pragma unroll
                for (int L = 0; L < S; ++L) {
                    uint32_t acc[8];
                    __syncwarp();  // tcgen05.ld is warp-collective
                    tmem_ld_32x32b_x8(lane_base + q * TN * S + TN * L + 8 * h, acc);
                    tmem_ld_wait();
                    const int sh = b * (S - 1 - L) - D;  // compile-time after unrolling
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const long long sL = (long long)__float2int_rn(__uint_as_float(acc[c]));
                        if (sh >= 0) T[c] += sL * (1ll << sh);
                        else T[c] += (sL + (1ll << (-sh - 1))) >> (-sh);
                    }
                }
                if (!rowok) continue;
                const int64_t gx0 = X0 + q * TN + 8 * h;
                double *dst = out + gy * Ex;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int64_t gx = gx0 + c, ix = gx - rh;
                    if (ix >= nx || ix < p.band || nx - 1 - ix < p.band) continue;
                    const double r = (double)T[c];
                    const double v = exp_add ? (T[c] ? __longlong_as_double(__double_as_longlong(r) + sc_bits) : 0.0)
                                             : r * s1 * s2;
                    dst[gx] = nan_tile ? __longlong_as_double(0x7FF8000000000000ll) : v;
                }
            }
        };

        int k = 0, prev = -1, prev_emax = 1;
        if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x);
        bool ok = true;
        for (int id = blockIdx.x; id < ntiles; id += gridDim.x, ++k) {
            const int bf = k & 1;
            const int emax = tile_emax(k);
            if (emax < 0) {
                ok = false;
                break;
            }
            // buffer bf was last read by the MMAs of tile k-2, whose completion
            // the epilogue of tile k-2 (previous iteration) waited for
            cut(A[bf], emax);
            fence_proxy_async_smem();
            mbar_arrive(&full[bf]);
            const int nid = id + gridDim.x;
            if (nid < ntiles) prefetch(nid);  // loads in flight during the epilogue
            if (k >= 1) {
                if (!bounded_wait(&done[bf ^ 1], ((k - 1) >> 1) & 1, kWaitCycles)) {
                    ok = false;
                    break;
                }
                fence_after_thread_sync();
                epilogue(prev, bf ^ 1, prev_emax);
                fence_before_thread_sync();
                mbar_arrive(&freeb[bf ^ 1]);
            }
            prev = id;
            prev_emax = emax;
        }
        if (ok && prev >= 0) {
            const int lb = (k - 1) & 1;
            ok = bounded_wait(&done[lb], ((k - 1) >> 1) & 1, kWaitCycles);
            fence_after_thread_sync();
            // test hook: the barrier's next phase is never completed
            if (ok && p.debug_unmet) ok = bounded_wait(&done[lb], (((k - 1) >> 1) & 1) ^ 1, kDebugWaitCycles);
            if (ok) epilogue(prev, lb, prev_emax);
        }
        if (!ok) atomicExch(abort_flag, 1);
    }
    fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *(volatile int *)abort_flag) atomicExch(&g_split_error, 1);
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

}  // namespace split
}  // namespace gbs

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace gbs {

namespace {

// Balanced digits of an integer (top first): V = sum_i d_i 2^(b(S-1-i)),
// |d_i| <= 2^(b-1) (the same cut the kernel makes on the device).
void host_digits(long long V, int b, int S, int *d)
{
    const long long half = 1ll << (b - 1), mask = (1ll << b) - 1;
    for (int i = S - 1; i >= 1; --i) {
        const long long di = ((V & mask) ^ half) - half;
        d[i] = (int)di;
        V = (V - di) >> b;
    }
    d[0] = (int)V;
}

int digit_bits(int S) { return S == 6 ? 9 : (S == 7 ? 8 : 7); }

}  // namespace

// The digit split of the composite kernel w^(t): the smallest S in {6, 7}
// (b = 9, 8 bits per digit, NB = S b - 1 >= 53 fixed-point bits) for which
// every level L = i + j < S of the products a_i b_j keeps its sum of absolute
// values below 2^24 for any input digits |a_i| <= 2^(b-1):
//   2^(b-1) * sum_{j <= L} sum_taps |b_j| < 2^24,
// so that FP32 accumulation of the level is exact.  Fills the digits, the
// K-block ranges and the result scale; UNSUPPORTED if no S qualifies or the
// fused radius exceeds 8.
stencil_status split_fill(const Plan &p, int t, split::SplitParams *sp, int *S_out)
{
    using namespace split;
    const int r = p.pat.r, R = t * r;
    if (p.pat.d != 2 || p.dtype != STENCIL_F64)
        return fail(STENCIL_ERR_UNSUPPORTED, "split FP64 path: 2-D FP64 grids only");
    if (R > kMaxR) return fail(STENCIL_ERR_UNSUPPORTED, "split FP64 path: fused radius t*r must be <= 8");
    const std::vector<double> wt = compose_dense(p.pat, p.w, t);
    const int lines = 2 * R + 1, taps = lines * lines;
    double wmax = 0;
    for (double x : wt) wmax = std::max(wmax, std::fabs(x));
    std::memset(sp, 0, sizeof(*sp));
    int Ew = 0;
    if (wmax > 0) std::frexp(wmax, &Ew);  // wmax < 2^Ew
    for (int S = 6; S <= kMaxS; ++S) {
        const int b = digit_bits(S), NB = S * b - 1;
        std::vector<int> dig((size_t)S * taps);
        for (int k = 0; k < taps; ++k) {
            const long long V = std::llround(std::ldexp(wt[k], NB - Ew));
            int d[kMaxS];
            host_digits(V, b, S, d);
            for (int j = 0; j < S; ++j) dig[(size_t)j * taps + k] = d[j];
        }
        bool ok = true;
        double cum = 0;  // sum over j <= L of sum_taps |b_j|
        for (int L = 0; L < S && ok; ++L) {
            for (int k = 0; k < taps; ++k) cum += std::abs(dig[(size_t)L * taps + k]);
            if (std::ldexp(cum, b - 1) >= 16777216.0) ok = false;
        }
        if (!ok) continue;
        for (int j = 0; j < S; ++j)
            for (int k = 0; k < taps; ++k) sp->wd[j][k] = (short)dig[(size_t)j * taps + k];
        const int D = std::max(0, 24 + b * (S - 1) - 62);
        sp->scale0 = b * (S - 1) + D + Ew - 2 * NB - 1022;
        *S_out = S;
        // K blocks of 16 window columns per line: line a is non-zero on
        // window columns [R - h_a, R + h_a + 15]
        for (int a = -R; a <= R; ++a) {
            const int h = composite_half(p.pat.shape, r, t, a);
            const int i = a + R;
            if (h < 0) {
                sp->kb_lo[i] = 1;
                sp->kb_hi[i] = 0;
                continue;
            }
            sp->kb_lo[i] = (unsigned char)((R - h) / KI);
            sp->kb_hi[i] = (unsigned char)std::min(kNkb - 1, (R + h + TN - 1) / KI);
        }
        sp->R = R;
        sp->rh = r;
        sp->band = (t - 1) * r;
        sp->hs = (TM + 2 * R) | 1;  // odd chunk-column height: conflict-free 16-byte staging stores
        sp->debug_unmet = p.debug_unmet_wait;
        sp->Ey = p.ext[1];
        sp->Ex = p.ext[2];
        return STENCIL_OK;
    }
    return fail(STENCIL_ERR_UNSUPPORTED, "split FP64 path: the composite weights' digit sums exceed the exact "
                                         "FP32 range at every digit width");
}

int split_slices(const Plan &p, int t)
{
    split::SplitParams sp;
    int S = 0;
    const std::string keep = stencil_last_error();  // a query: leave the last error as it was
    if (split_fill(p, t, &sp, &S) != STENCIL_OK) S = 0;
    fail(STENCIL_OK, keep);
    return S;
}

// Column blocks of 16 per tile that fit in 227 KB of shared memory with
// double-buffered digit slices: 2 if they fit, else 1 (0: none fits).
int split_nacc(int R, int S)
{
    const int hs = (split::TM + 2 * R) | 1;
    for (int nacc = 2; nacc >= 1; --nacc) {
        const int nch = 2 * nacc + 2;
        const size_t a_bytes = (size_t)S * nch * hs * 16;
        const size_t b_bytes = (size_t)(2 * R + 1) * split::kNkb * 2 * S * 256;
        if (split::kHeader + b_bytes + 2 * a_bytes <= 227 * 1024) return nacc;
    }
    return 0;
}

namespace {

template <int S, int NACC>
stencil_status launch_split_n(const Plan &p, const split::SplitParams &sp, const void *in, void *out,
                              cudaStream_t st)
{
    using namespace split;
    SplitParams tp = sp;
    tp.nch = 2 * NACC + 2;
    const size_t a_bytes = (size_t)S * tp.nch * tp.hs * 16;
    const size_t b_bytes = (size_t)(2 * tp.R + 1) * kNkb * 2 * S * 256;
    const size_t smem = kHeader + b_bytes + 2 * a_bytes;
    auto kern = tc2d_split<S, NACC>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t TX = NACC * TN;
    const int64_t nty = (p.dims[1] + TM - 1) / TM, ntx = (p.dims[2] + TX - 1) / TX;
    const int64_t ntiles = nty * ntx;
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
    // staged windows start at column X0 - R = (r - R) + 32 tx: 16-byte loads
    // when that is even, the stored rows are 16-byte multiples and `in` is
    // 16-byte aligned
    tp.vec16 = ((p.pat.r - tp.R) % 2 == 0) && (p.ext[2] % 2 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
    kern<<<grid, kThreads, smem, st>>>((const double *)in, (double *)out, tp, (int)ntiles, (int)ntx);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "tc2d_split launch");
}

}  // namespace

stencil_status read_split_error(int *flag)
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_split_error, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_split_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the split kernel's error word");
    *flag = v;
    return STENCIL_OK;
}

stencil_status launch_split_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    split::SplitParams sp;
    int S = 0;
    stencil_status s = split_fill(p, t, &sp, &S);
    if (s != STENCIL_OK) return s;
    const int nacc = split_nacc(sp.R, S);
    if (S == 6 && nacc == 2) s = launch_split_n<6, 2>(p, sp, in, out, st);
    else if (S == 6 && nacc == 1) s = launch_split_n<6, 1>(p, sp, in, out, st);
    else if (S == 7 && nacc == 2) s = launch_split_n<7, 2>(p, sp, in, out, st);
    else if (S == 7 && nacc == 1) s = launch_split_n<7, 1>(p, sp, in, out, st);
    else return fail(STENCIL_ERR_UNSUPPORTED, "split FP64 path: tile does not fit in shared memory");
    if (s != STENCIL_OK || t == 1) return s;
    // points within (t-1) r of the boundary: stepwise on CUDA cores
    return launch_cu_band(p, in, out, t, (t - 1) * p.pat.r, st);
}

}  // namespace gbs
