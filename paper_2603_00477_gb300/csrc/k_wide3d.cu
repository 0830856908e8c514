// k_wide3d.cu -- 3-D FP32 grids on the FP16 tensor cores (precision f16, one
// step per sweep): the operand-exchanged Toeplitz formulation of k_wide.cu,
// marched along z.
//
// One output plane z of a 3-D sweep is the sum over the lines (dz, dy) of
// the stencil of 1-D Toeplitz products along x (paper Sec. 2.2 applied per
// line): out[z][y][x] = sum_(dz,dy) sum_dx w[dz][dy][dx] u[z+dz][y+dy][x+dx].
// As in the 2-D wide kernel, line (dz, dy)'s Toeplitz factor is the A operand
// (M = 128 output columns in reverse order, one strip of core matrices per
// line that every K block reads through LBO = SBO = 128 bytes) and the staged
// input plane z + dz is the B operand (N = NR output rows: the descriptor
// starts at row dy + R of the plane's chunk-column tile).
//
// A CTA takes a stack of NR x 128 tiles and marches it through a run of
// planes.  Input plane p of the run is staged once, into slot p mod S of a
// ring of S = 2R + 2 slots, and read by the MMAs of the 2R + 1 output planes
// whose window holds it; the loaders stage the plane that completes output
// plane z's window while the MMAs of z - 1 run.
//
// Scaling: each staged plane tile gets its own power-of-two scale 2^es_p
// (es_p = 141 - its largest exponent, so |x| 2^es_p < 2^15).  For output
// plane z, c = min es_p over its 2R + 1 planes; the strip of line (dz, dy) is
// written with the weights scaled by 2^(15 - ew + c - es_(z+dz)), a power of
// two <= 2^(15 - ew), so every product carries the common factor
// 2^(15 - ew + c) and the epilogue multiplies by 2^(ew - 15 - c).  The strips
// are double-buffered and only their non-zero core matrices are rewritten per
// output plane.
//
// Roles (800 threads, one CTA per SM): warps 0-15 stage planes (pass 1: the
// tile's largest |x|, exchanged through an mbarrier; pass 2: scale, convert
// to FP16, store in the chunk-column layout) and write the strips; one
// thread of warp 24 issues the MMAs into two TMEM accumulators of NR
// columns; warps 16-23 drain them (one output column per thread, 32
// consecutive columns per warp store).  Every wait is bounded.
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

// Set when a bounded wait of this kernel runs out.
__device__ int g_wide3_error;

namespace wide3 {

using namespace tc;

constexpr int kMaxR = 3;
constexpr int kSide = 2 * kMaxR + 1;
constexpr int kMaxLines = kSide * kSide;  // (dz, dy) pairs
constexpr int TM = 128;                   // output columns per tile (MMA M)
constexpr int kLoadWarps = 16;            // warps 0-15
constexpr int kLoaders = 32 * kLoadWarps;
constexpr int kEpiWarp = kLoadWarps;      // warps 16-23
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = kLoadWarps + kEpiWarps;  // warp 24
constexpr int kThreads = 32 * (kMmaWarp + 1);
constexpr int kConv = 10;  // independent 16-byte loads in flight per loader thread
constexpr int kHeader = 1024;
constexpr unsigned long long kWaitCycles = 4ull << 30;       // ~2 s at 2 GHz
constexpr unsigned long long kDebugWaitCycles = 1ull << 22;  // ~2 ms: the test hook's limit

struct Wide3Params {
    double w[kMaxLines * kSide];  // per line: its 2R+1 weights along x (dx = -R .. R)
    signed char ldz[kMaxLines], ldy[kMaxLines];
    unsigned char kb_lo[kMaxLines], kb_hi[kMaxLines];
    int nlines, R, nkb, hs, delta, ew, S, zrun, nzc, ntx, nty;
    int debug_unmet;  // test hook: wait once more on an mbarrier phase that never completes
    int vec;          // values per load: 4 (16 bytes) or 2 (8 bytes) when stored rows are multiples of
                      // that many bytes (tiles then start aligned), else 1
    int xshift;       // tiles start xshift columns left of column 0
    int64_t Ez, Ey, Ex;
};

__device__ __forceinline__ float pow2f(int e)  // 2^e for -126 <= e <= 127
{
    return __int_as_float((e + 127) << 23);
}


template <int NR, int NKB>
__global__ void __launch_bounds__(kThreads, 1)
    tc3d_wide(const float *__restrict__ in, float *__restrict__ out, const __grid_constant__ Wide3Params p, int nruns)
{
    constexpr uint32_t kCols = 2 * NR;  // two accumulators of NR columns
    static_assert(kCols <= 512, "TMEM columns");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem);
    int *abort_flag = reinterpret_cast<int *>(smem + 4);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 16);     // [2] window of an output plane staged
    uint64_t *done = reinterpret_cast<uint64_t *>(smem + 32);     // [2] MMAs of an output plane complete
    uint64_t *accfree = reinterpret_cast<uint64_t *>(smem + 48);  // [2] accumulator drained
    uint64_t *maxb = reinterpret_cast<uint64_t *>(smem + 64);     // [2] exponent exchange
    uint64_t *eub = reinterpret_cast<uint64_t *>(smem + 80);      // [4] an output plane's scale published
    int *wmax = reinterpret_cast<int *>(smem + 128);              // [2][kLoadWarps]
    int *eus = reinterpret_cast<int *>(smem + 256);               // [4] scale exponent c per output plane
    int *es_ring = reinterpret_cast<int *>(smem + 288);           // [S] scale exponent per staged slot
    float *wsc = reinterpret_cast<float *>(smem + 512);           // [nlines][2R+1] FP16 weights x 2^(15-ew)
    constexpr int nkb = NKB;
    const int R = p.R, HS = p.hs, S = p.S, nlines = p.nlines;
    const uint32_t strip_bytes = (uint32_t)((nlines - 1) * p.delta + 2 * nkb + 15) * 128;
    const uint32_t in_bytes = (uint32_t)(2 * nkb) * HS * 16;
    unsigned char *Wbase = smem + kHeader;                // strip sets 0 and 1
    unsigned char *ibase = Wbase + 2 * strip_bytes;       // S input slots
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t Ez = p.Ez, Ey = p.Ey, Ex = p.Ex, plane = Ey * Ex;

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
    // both strip sets: zero them once (only the non-zero core matrices change)
    for (uint32_t i = (uint32_t)tid * 16; i < 2 * strip_bytes; i += kThreads * 16)
        *reinterpret_cast<uint4 *>(Wbase + i) = make_uint4(0, 0, 0, 0);
    // the weights scaled by 2^(15 - ew) (|w| 2^(15-ew) < 2^15) and rounded to
    // FP16 once; each output plane rescales them by exact powers of two
    for (int i = tid; i < nlines * (2 * R + 1); i += kThreads)
        wsc[i] = __half2float(__double2half(ldexp(p.w[i], 15 - p.ew)));
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
    // run -> stack (rows Y0.., columns X0..) and output planes zbeg .. zbeg + nout - 1
    auto run_of = [&](int run, int64_t *Y0, int64_t *X0, int64_t *zbeg, int *nout) {
        const int stack = run / p.nzc, zc = run - stack * p.nzc;
        *Y0 = R + (int64_t)(stack / p.ntx) * NR;
        *X0 = (int64_t)(stack % p.ntx) * TM - p.xshift;
        *zbeg = R + (int64_t)zc * p.zrun;
        *nout = (int)min((int64_t)p.zrun, Ez - R - *zbeg);
    };

    if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kFmtF16, TM, NR);
            int k = 0, qs = 0;  // output planes / staged planes so far
            bool ok = true;
            for (int run = blockIdx.x; run < nruns && ok; run += gridDim.x) {
                int64_t Y0, X0, zbeg;
                int nout;
                run_of(run, &Y0, &X0, &zbeg, &nout);
                for (int o = 0; o < nout; ++o, ++k) {
                    const int b = k & 1;
                    if (!bounded_wait(&full[b], (k >> 1) & 1, kWaitCycles)) {
                        ok = false;
                        break;
                    }
                    if (k >= 2 && !bounded_wait(&accfree[b], ((k - 2) >> 1) & 1, kWaitCycles)) {
                        ok = false;
                        break;
                    }
                    fence_after_thread_sync();
                    const uint64_t a0 = smem_desc(smem_u32(Wbase + b * strip_bytes), 128, 128);
                    const uint32_t d = tmem + (uint32_t)(b * NR);
                    uint32_t acc = 0;
                    for (int l = 0; l < nlines; ++l) {
                        const int klo = p.kb_lo[l], khi = p.kb_hi[l];
                        // input plane of this line: run-local staged index o + R + dz
                        const int slot = (qs + o + R + p.ldz[l]) % S;
                        const uint64_t b0 = smem_desc(smem_u32(ibase + slot * in_bytes), (uint32_t)HS * 16, 128);
                        uint64_t da = a0 + (uint64_t)(l * p.delta + 2 * klo) * 8;
                        uint64_t db = b0 + (uint64_t)(2 * klo) * HS + (uint64_t)(p.ldy[l] + R);
                        for (int kb = klo; kb <= khi; ++kb) {
                            mma_f16(d, da, db, idesc, acc);
                            acc = 1;
                            da += 16;
                            db += (uint64_t)(2 * HS);
                        }
                    }
                    mma_commit(&done[b]);
                }
                qs += nout + 2 * R;
            }
            // the last output planes' MMAs complete before the TMEM is released
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
        const int vec = p.vec;
        const int jn = (127 + 2 * R) / 8 - 15 + 1;  // non-zero core matrices of a strip: 15 .. 15 + jn - 1
        int k = 0, qs = 0;
        bool ok = true;
        // the shifts each strip set was last written with (none yet)
        uint64_t set_sig[2] = {~0ull, ~0ull};
        int es_guess = 0;  // the scale exponent of the last plane converted
        for (int run = blockIdx.x; run < nruns && ok; run += gridDim.x) {
            int64_t Y0, X0, zbeg;
            int nout;
            run_of(run, &Y0, &X0, &zbeg, &nout);
            const int kbase = k;
            // the slots still hold planes of the previous run: its MMAs must be done
            if (kbase >= 1 && !bounded_wait(&done[(kbase - 1) & 1], ((kbase - 1) >> 1) & 1, kWaitCycles)) break;
            const bool rows_in = vec > 1 && Y0 - R >= 0 && Y0 - R + rows <= Ey && X0 - R >= 0 &&
                                 X0 - R + 16 * NKB <= Ex;
            const int P = nout + 2 * R;  // planes this run stages
            const float *pin0 = in + (zbeg - R) * plane;  // its first plane (inside [0, Ez))
            // item i (row r, 4-value column c) of the plane tile at pl; cells
            // outside the stored array read as zero
            auto load = [&](const float *pl, int i, int r, int c) -> float4 {
                if (rows_in) {
                    const float *a = pl + (Y0 - R + r) * Ex + (X0 - R) + 4 * c;
                    if (vec == 4) return __ldcg(reinterpret_cast<const float4 *>(a));
                    const float2 lo = __ldcg(reinterpret_cast<const float2 *>(a));
                    const float2 hi = __ldcg(reinterpret_cast<const float2 *>(a + 2));
                    return make_float4(lo.x, lo.y, hi.x, hi.y);
                }
                const int64_t gy = Y0 - R + i / F4, gx = X0 - R + 4 * (i % F4);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (gy < 0 || gy >= Ey) return v;
                const float *g = pl + gy * Ex;
                if (vec == 4) {
                    // X0 - R is a multiple of 4: the 4 values lie wholly inside or outside the row
                    if (gx >= 0 && gx < Ex) v = __ldcg(reinterpret_cast<const float4 *>(g + gx));
                    return v;
                }
                if (vec == 2) {
                    // X0 - R and Ex are even: each pair lies wholly inside or outside the row
                    if (gx >= 0 && gx < Ex) {
                        const float2 a = __ldcg(reinterpret_cast<const float2 *>(g + gx));
                        v.x = a.x;
                        v.y = a.y;
                    }
                    if (gx + 2 >= 0 && gx + 2 < Ex) {
                        const float2 a = __ldcg(reinterpret_cast<const float2 *>(g + gx + 2));
                        v.z = a.x;
                        v.w = a.y;
                    }
                    return v;
                }
                if (gx >= 0 && gx < Ex) v.x = __ldcg(g + gx);
                if (gx + 1 >= 0 && gx + 1 < Ex) v.y = __ldcg(g + gx + 1);
                if (gx + 2 >= 0 && gx + 2 < Ex) v.z = __ldcg(g + gx + 2);
                if (gx + 3 >= 0 && gx + 3 < Ex) v.w = __ldcg(g + gx + 3);
                return v;
            };
            auto absmax4 = [](unsigned m, float4 v) -> unsigned {
                return max(m, max(max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu),
                                  max(__float_as_uint(v.z) & 0x7fffffffu, __float_as_uint(v.w) & 0x7fffffffu)));
            };
            // the exponent exchange of staged plane q (counter): every loader gets
            // es = 141 - the tile's largest exponent, clamped (|x| 2^es < 2^15)
            auto exchange = [&](unsigned mxu, int q, int *es_out) -> bool {
                const int qb = q & 1;
                const int mx = (int)(__reduce_max_sync(0xffffffffu, mxu) >> 23);
                if (lane == 0) wmax[qb * kLoadWarps + warp] = mx;
                __syncwarp();
                mbar_arrive(&maxb[qb]);
                if (!bounded_wait(&maxb[qb], (q >> 1) & 1, kWaitCycles)) return false;
                int emax = wmax[qb * kLoadWarps];
#pragma unroll
                for (int w = 1; w < kLoadWarps; ++w) emax = max(emax, wmax[qb * kLoadWarps + w]);
                *es_out = max(-126, min(127, 141 - emax));
                return true;
            };
            for (int j = 0; j < P && ok; ++j) {
                const int q = qs + j, slot = q % S;
                const float *pin = pin0 + (int64_t)j * plane;
                // ask L2 for the next plane while this one is read
                if (j + 1 < P) {
                    const float *pf = pin + plane;
                    const int64_t gx_lo = max((int64_t)0, X0 - R), gx_hi = min(Ex, X0 - R + 16 * NKB);
                    if (gx_lo < gx_hi) {
                        const int nl = (int)((gx_hi - gx_lo + 31) / 32);
                        for (int e = tid; e < rows * nl; e += kLoaders) {
                            const int row = e / nl, l = e - (e / nl) * nl;
                            const int64_t gy = Y0 - R + row;
                            if (gy < 0 || gy >= Ey) continue;
                            const int64_t gx = min(gx_lo + 32 * (int64_t)l, gx_hi - 1);
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(pf + gy * Ex + gx));
                        }
                    }
                }
                // the slot's previous plane (run-local j - S) was last read by
                // output plane j - S; from an earlier run, it is covered by the
                // wait at the start of the run
                const int o_done = j - S;
                if (o_done >= 0 && !bounded_wait(&done[(kbase + o_done) & 1], ((kbase + o_done) >> 1) & 1,
                                                 kWaitCycles)) {
                    ok = false;
                    break;
                }
                // one pass: scale by the previous plane's 2^es (a guess), convert and
                // store 4 FP16 values (8 bytes) per float4, and take the largest |x|
                unsigned char *hi = ibase + slot * in_bytes;
                auto convert = [&](float xs, unsigned *mxu) {
                    // kConv items in flight per thread: one round trip for a
                    // 128-row tile at r = 1 (130 x 36 items over 512 threads)
                    for (int i0 = tid; i0 < items; i0 += kConv * kLoaders) {
                        float4 vb[kConv];
#pragma unroll
                        for (int u = 0; u < kConv; ++u) {
                            const int i = i0 + u * kLoaders;
                            vb[u] = i < items ? load(pin, i, i / F4, i % F4) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < kConv; ++u) {
                            const int i = i0 + u * kLoaders;
                            if (i >= items) break;
                            const float4 v = vb[u];
                            const int rr = i / F4, cc = i % F4;
                            *mxu = absmax4(*mxu, v);
                            const __half2 h01 = __floats2half2_rn(v.x * xs, v.y * xs);
                            const __half2 h23 = __floats2half2_rn(v.z * xs, v.w * xs);
                            const uint32_t off = (uint32_t)((cc >> 1) * HS + rr) * 16 + (uint32_t)(cc & 1) * 8;
                            uint2 hv;
                            hv.x = *reinterpret_cast<const uint32_t *>(&h01);
                            hv.y = *reinterpret_cast<const uint32_t *>(&h23);
                            *reinterpret_cast<uint2 *>(hi + off) = hv;
                        }
                    }
                };
                unsigned mxu = 0;
                int es = es_guess;
                convert(pow2f(es), &mxu);
                int es_exact = 0;
                if (!exchange(mxu, q, &es_exact)) {
                    ok = false;
                    break;
                }
                // the guess is kept when no value overflowed (es <= es_exact) and
                // the tile's largest value keeps at least 2^7 of the FP16 range
                // (es >= es_exact - 8); else convert again with the exact scale
                // (every loader decides alike)
                if (es > es_exact || es < es_exact - 8) {
                    es = es_exact;
                    unsigned unused = 0;
                    convert(pow2f(es), &unused);
                }
                es_guess = es;
                // every loader holds es; tid 0 also records it for the output
                // planes to come (read after a later exchange barrier)
                if (tid == 0) es_ring[slot] = es;
                fence_proxy_async_smem();
                if (j >= 2 * R) {
                    // plane j completes the window of output plane o = j - 2R (counter kk)
                    const int o = j - 2 * R, kk = kbase + o, b = kk & 1;
                    // c over planes o .. o + 2R: the earlier ones from es_ring, plane j
                    // from this thread's es; the shift of line (dz, dy) is c - es of
                    // plane o + R + dz
                    int c = es;
                    for (int i = 0; i < 2 * R; ++i) c = min(c, es_ring[(qs + o + i) % S]);
                    uint64_t sig = 0;  // the 2R + 1 shifts, 7 bits each
                    for (int i = 0; i <= 2 * R; ++i) {
                        const int e_i = i == 2 * R ? es : es_ring[(qs + o + i) % S];
                        sig |= (uint64_t)(-max(-126, c - e_i)) << (7 * i);
                    }
                    // strip set b was last read by the MMAs of output kk - 2 (waited
                    // for above: j - S = o - 2); it needs rewriting only if its shifts
                    // changed (every loader decides alike from the same values)
                    if (sig != set_sig[b]) {
                        set_sig[b] = sig;
                        unsigned char *W = Wbase + b * strip_bytes;
                        const int side = 2 * R + 1;
                        for (int e = tid; e < nlines * jn * 64; e += kLoaders) {
                            const int ii = (e >> 3) & 7, jj = e & 7, rest = e >> 6;
                            const int J = 15 + rest % jn, l = rest / jn;
                            const int idx = 8 * J + ii + jj - 127;  // dx + R of output column 127 - (8g + ii)
                            if (idx < 0 || idx > 2 * R) continue;
                            const int sh = -(int)((sig >> (7 * (R + p.ldz[l]))) & 127);
                            // FP16 weight x 2^sh, sh <= 0: exact unless it falls below
                            // FP16's normal range (a plane 2^14 times smaller than the largest)
                            const __half hv = __float2half_rn(wsc[l * side + idx] * pow2f(sh));
                            const uint32_t off = (uint32_t)(l * p.delta + J) * 128 + ii * 16 + jj * 2;
                            *reinterpret_cast<__half *>(W + off) = hv;
                        }
                        fence_proxy_async_smem();
                    }
                    // publish the scale: slot kk & 3 was last read by the epilogue of
                    // output kk - 4, which finished before the MMAs of kk - 2 started
                    if (tid == 0) {
                        eus[kk & 3] = c;
                        mbar_arrive(&eub[kk & 3]);
                    }
                    mbar_arrive(&full[b]);
                }
            }
            k += nout;
            qs += nout + 2 * R;
        }
    } else {
        // ---------------- epilogue (warps 16-23) ----------------
        const int q4 = (warp - kEpiWarp) & 3, h = (warp - kEpiWarp) >> 2;
        const int m = TM - 1 - (32 * q4 + lane);
        const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16);
        int k = 0;
        bool ok = true;
        for (int run = blockIdx.x; run < nruns && ok; run += gridDim.x) {
            int64_t Y0, X0, zbeg;
            int nout;
            run_of(run, &Y0, &X0, &zbeg, &nout);
            const int64_t gx = X0 + m;
            const bool colok = gx >= R && gx < Ex - R;
            // rows n of the tile written: interior rows Y0 + n < Ey - R
            const int n_hi = (int)min((int64_t)NR, Ey - R - Y0);
            for (int o = 0; o < nout; ++o, ++k) {
                const int b = k & 1;
                if (!bounded_wait(&eub[k & 3], (k >> 2) & 1, kWaitCycles)) {
                    ok = false;
                    break;
                }
                const int c = eus[k & 3];
                if (!bounded_wait(&done[b], (k >> 1) & 1, kWaitCycles)) {
                    ok = false;
                    break;
                }
                fence_after_thread_sync();
                // out = acc 2^(ew - 15 - c), as two in-range powers of two
                const int e = p.ew - 15 - c, e1 = e / 2, e2 = e - e1;
                const float s1 = pow2f(max(-126, min(127, e1))), s2 = pow2f(max(-126, min(127, e2)));
                float *op = out + (zbeg + o) * plane + Y0 * Ex + gx;
                for (int n0 = h * (NR / 2); n0 < (h + 1) * (NR / 2); n0 += 16) {
                    uint32_t v[16];
                    __syncwarp();
                    tmem_ld_32x32b_x16(lane_base + (uint32_t)(b * NR + n0), v);
                    tmem_ld_wait();
                    if (n0 >= n_hi) break;  // rows below the interior
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int n = n0 + jj;
                        if (colok && n < n_hi) op[(int64_t)n * Ex] = __uint_as_float(v[jj]) * s1 * s2;
                    }
                }
                fence_before_thread_sync();
                mbar_arrive(&accfree[b]);
            }
        }
        if (ok && p.debug_unmet && k > 0) {
            // test hook: a phase that never completes -> the bounded wait reports it
            bounded_wait(&done[(k - 1) & 1], (((k - 1) >> 1) & 1) ^ 1, kDebugWaitCycles);
        }
    }
    fence_before_thread_sync();
    __syncthreads();
    if (tid == 0 && *(volatile int *)abort_flag) atomicExch(&g_wide3_error, 1);
    if (warp == kMmaWarp) tmem_dealloc(tmem, kCols);
}

}  // namespace wide3

namespace {

template <int NR>
stencil_status launch_wide3_n(const Plan &p, const void *in, void *out, cudaStream_t st)
{
    using namespace wide3;
    const int R = p.pat.r, side = 2 * R + 1;
    if (R > kMaxR) return fail(STENCIL_ERR_UNSUPPORTED, "3-D wide FP16 path: r must be <= 3");
    // lines (dz, dy) with a non-zero tap of the pattern, lexicographic; the
    // half-width of each is its largest |dx|
    int half[kSide][kSide];
    for (auto &row : half)
        for (int &h : row) h = -1;
    for (int k = 0; k < p.pat.K; k++) {
        const int dz = p.pat.offs[3 * k], dy = p.pat.offs[3 * k + 1], dx = p.pat.offs[3 * k + 2];
        int &h = half[dz + R][dy + R];
        h = std::max(h, std::abs(dx));
    }
    const std::vector<double> wd = compose_dense(p.pat, p.w, 1);  // (2R+1)^3, (dz, dy, dx) lexicographic
    Wide3Params wp;
    std::memset(&wp, 0, sizeof(wp));
    const int nkb = (128 + 2 * R + 15) / 16;
    int nl = 0;
    double wmax = 0;
    for (int a = 0; a < side; a++)
        for (int b = 0; b < side; b++) {
            const int h = half[a][b];
            if (h < 0) continue;
            wp.ldz[nl] = (signed char)(a - R);
            wp.ldy[nl] = (signed char)(b - R);
            // non-zero window columns R - h .. R + h + 127 (tc_lines_2d's rule at M = 128, K = 16)
            wp.kb_lo[nl] = (unsigned char)((R - h) / 16);
            wp.kb_hi[nl] = (unsigned char)std::min(nkb - 1, (R + h + 127) / 16);
            for (int c = 0; c < side; c++) {
                const double v = wd[((size_t)a * side + b) * side + c];
                wp.w[nl * side + c] = v;
                wmax = std::max(wmax, std::fabs(v));
            }
            nl++;
        }
    if (nl != tc_wide3_lines(p.pat.shape, R)) return fail(STENCIL_ERR_INTERNAL, "3-D wide FP16 path: lines");
    if (nl * side > 128) return fail(STENCIL_ERR_UNSUPPORTED, "3-D wide FP16 path: too many weights");
    const Wide3Geom g = tc_wide3_geom(R, nl, NR);
    if (g.smem > 227 * 1024) return fail(STENCIL_ERR_UNSUPPORTED, "3-D wide FP16 tile does not fit in shared memory");
    if (g.nkb != 9) return fail(STENCIL_ERR_INTERNAL, "3-D wide FP16 path: K blocks");
    wp.nlines = nl;
    wp.R = R;
    wp.nkb = g.nkb;
    wp.hs = g.hs;
    wp.delta = g.delta;
    wp.S = g.slots;
    wp.ew = 0;
    if (wmax > 0) std::frexp(wmax, &wp.ew);  // wmax < 2^ew
    wp.debug_unmet = p.debug_unmet_wait;
    wp.Ez = p.ext[0];
    wp.Ey = p.ext[1];
    wp.Ex = p.ext[2];
    const uintptr_t addr = reinterpret_cast<uintptr_t>(in);
    wp.vec = (p.ext[2] % 4 == 0 && addr % 16 == 0) ? 4 : (p.ext[2] % 2 == 0 && addr % 8 == 0) ? 2 : 1;
    wp.xshift = (wp.vec - R % wp.vec) % wp.vec;  // (tile start - R) a multiple of vec
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t nz = p.dims[0];
    wp.nty = (int)((p.dims[1] + NR - 1) / NR);
    wp.ntx = (int)((p.ext[2] + wp.xshift + TM - 1) / TM);
    const int64_t stacks = (int64_t)wp.nty * wp.ntx;
    // run length: the fewest rounds of resident CTAs times the planes a run
    // stages (its outputs + 2R)
    int64_t best_z = nz;
    double best = 1e300;
    for (int64_t cz = 1; cz <= nz; cz++) {
        const int64_t runs = stacks * ((nz + cz - 1) / cz);
        const double cost = (double)((runs + sms - 1) / sms) * (double)(cz + 2 * R);
        if (cost < best) {
            best = cost;
            best_z = cz;
        }
    }
    wp.zrun = (int)best_z;
    wp.nzc = (int)((nz + best_z - 1) / best_z);
    const int64_t nruns = stacks * wp.nzc;
    if (nruns > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    auto kern = tc3d_wide<NR, 9>;
    stencil_status s = ensure_smem((const void *)kern, g.smem);
    if (s != STENCIL_OK) return s;
    const unsigned grid = (unsigned)std::min<int64_t>(nruns, sms);
    kern<<<grid, kThreads, g.smem, st>>>((const float *)in, (float *)out, wp, (int)nruns);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "tc3d_wide launch");
}

}  // namespace

stencil_status launch_wide3_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.pat.d != 3 || p.dtype != STENCIL_F32 || t != 1)
        return fail(STENCIL_ERR_UNSUPPORTED, "3-D wide FP16 path: FP32 grids, one step per sweep");
    switch (tc_wide3_nrows(p.pat.shape, p.pat.r)) {
    case 128: return launch_wide3_n<128>(p, in, out, st);
    case 64: return launch_wide3_n<64>(p, in, out, st);
    case 32: return launch_wide3_n<32>(p, in, out, st);
    default: return fail(STENCIL_ERR_UNSUPPORTED, "3-D wide FP16 tile does not fit in shared memory");
    }
}

stencil_status read_wide3_error(int *flag)
{
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_wide3_error, sizeof(int));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_wide3_error, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the 3-D wide kernel's error word");
    *flag = v;
    return STENCIL_OK;
}

}  // namespace gbs
