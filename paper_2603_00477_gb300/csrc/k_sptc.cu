// k_sptc.cu -- the 2:4-structured sparse tensor-core sweep (paper Sec. 4.3):
// the t-step composite stencil as banded Toeplitz products on the sparse MMA,
// mma.sp m16n8k16 TF32 (1:2 sparsity of the A operand per pair of K).
//
// The Toeplitz block of a line of w^(t) is the sparse A operand (M = 16
// output columns, logical K = the permuted input window); B is the im2col of
// the staged input (N = 8 output rows).  The K permutation, the compressed
// values and their selectors follow sp_layout_2d / sp_a_value, which the
// dispatcher also uses to report S.
//
// CTA: 256 threads, tile 128 output rows x 64 output columns, persistent over
// tiles; the next tile's input is copied (cp.async: 16-byte copies when the
// stored rows are 16-byte multiples, the tile grid then shifted so each
// window starts on a 16-byte boundary) while this one computes, where two
// staging buffers fit; every thread rounds the elements it copied to TF32 in
// place.  Warp w owns the 16-column strip w mod 4 and the 64-row band w / 4.
// Its eight accumulators cover the rows y0 + 8n (y0 = 0..7, n = 0..7) of the
// band, so the B fragment of input row offset rho = y0 + a (line a) is shared
// by every (y0, a) with the same sum: a B fragment (one 16-byte shared-memory
// load per thread) feeds up to eight MMAs of different lines.  The compressed
// A fragments of all lines are built once per CTA in shared memory and held
// in registers for a pass of LC lines.
//
// Like the dense tensor-core sweeps it writes interior points farther than
// (t-1) r from the boundary; the CUDA-core band sweep computes the others.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "launch.h"
#include "tc_layout.h"

namespace gbs {

namespace {

constexpr int kSpMaxLines = 25;

struct SpParams {
    double w[kSpMaxLines * kSpMaxLines];  // composite w^(t), (2R+1)^2, row-major
    int cf[2 * kSpMaxNs], cs[2 * kSpMaxNs], bchunk[4 * kSpMaxNs];
    unsigned char mask[kSpMaxLines];
    int R, rh, band, lines, sigma, pitch_q, rl, nbuf;
    int vec16;  // 1: rows of the stored grid are 16-byte multiples and tiles start xshift columns left of
    int xshift; //    the interior so that every staged 16-byte chunk is aligned in global memory
    int64_t Ey, Ex;
};

__device__ __forceinline__ float cvt_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_sp(float (&d)[4], const float4 &a, const float4 &b, uint32_t e)
{
    asm volatile(
        "mma.sp::ordered_metadata.sync.aligned.m16n8k16.row.col.f32.tf32.tf32.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9,%10,%11}, {%0,%1,%2,%3}, %12, 0x0;"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)), "r"(__float_as_uint(a.w)),
          "r"(__float_as_uint(b.x)), "r"(__float_as_uint(b.y)), "r"(__float_as_uint(b.z)), "r"(__float_as_uint(b.w)),
          "r"(e));
}

__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gmem_src, bool valid)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(gmem_src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(float *smem_dst, const float *gmem_src, bool valid)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kSpTY = 128, kSpTX = 64;

// Fragment layout of mma.sp m16n8k16 TF32 (lane = 4 g + q):
//   A (16 x 8 compressed): a0 (row g, pair q), a1 (g+8, q), a2 (g, q+4),
//   a3 (g+8, q+4);  B (16 x 8 logical): b_j = B[q + 4j][g];
//   D: d0 (g, 2q), d1 (g, 2q+1), d2 (g+8, 2q), d3 (g+8, 2q+1);
//   selectors (selector 0: lanes with q < 2): lane 4g + h, nibble i ->
//   (row g, pair 4h + i), nibble 4 + i -> (row g + 8, pair 4h + i);
//   0x4 keeps the first member of the pair, 0xE the second.
// One pass over NL consecutive lines (a_lo .. a_lo+NL-1) of the composite:
// their compressed A fragments are held in registers; for each input row
// offset rho the B fragments (one 16-byte load per instruction) are loaded
// once, one row ahead, and fed to every (accumulator y0, line a) with
// y0 + a = rho.
template <int NS, int NL, bool FULL>
__device__ __forceinline__ void sp_pass(float (&acc)[8][4], const float *Tw, int a_lo, int RP, const int (&boff0)[NS],
                                        const int (&boff1)[NS], int g, const float4 *Af, const uint32_t *Em,
                                        const unsigned char *mask, int lane)
{
    float4 A[NL][NS];
    uint32_t E[NL][NS];
    unsigned mk[NL];
#pragma unroll
    for (int al = 0; al < NL; al++) {
        mk[al] = FULL ? 0xFu : mask[a_lo + al];
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const int idx = ((a_lo + al) * NS + s) * 32 + lane;
            A[al][s] = Af[idx];
            E[al][s] = Em[idx];
        }
    }
    auto loadB = [&](int rho, float4 (&Bv)[NS]) {
        const int swz = ((rho >> 3) ^ g) & 1;  // bit 3 of the staged row rho + 8 g
        const float *srow = Tw + (size_t)rho * RP;
#pragma unroll
        for (int s = 0; s < NS; s++) Bv[s] = *reinterpret_cast<const float4 *>(srow + (swz ? boff1[s] : boff0[s]));
    };
    float4 Bb[2][NS];  // row rr in Bb[rr & 1], row rr + 1 loaded ahead into the other
    loadB(a_lo, Bb[0]);
#pragma unroll
    for (int rr = 0; rr < NL + 7; rr++) {
        if (rr + 1 < NL + 7) loadB(a_lo + rr + 1, Bb[(rr + 1) & 1]);
#pragma unroll
        for (int s = 0; s < NS; s++) {
#pragma unroll
            for (int y0 = 0; y0 < 8; y0++) {
                const int al = rr - y0;
                if (al < 0 || al >= NL) continue;
                if (FULL || ((mk[al] >> s) & 1u)) mma_sp(acc[y0], A[al][s], Bb[rr & 1][s], E[al][s]);
            }
        }
    }
}

template <int NS, int LC, bool FULL>
__global__ void __launch_bounds__(256, 2) sptc2d_sweep(const float *__restrict__ in, float *__restrict__ out,
                                                       const __grid_constant__ SpParams p, int ntiles, int ntx)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int R = p.R, lines = p.lines, PQ = p.pitch_q;
    float4 *Af = reinterpret_cast<float4 *>(smem_raw);                  // [lines][NS][32]
    uint32_t *Em = reinterpret_cast<uint32_t *>(Af + lines * NS * 32);  // [lines][NS][32]
    float *S = reinterpret_cast<float *>(Em + lines * NS * 32);         // one or two staged tiles
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    const int ws = warp & 3, wb = warp >> 2;

    for (int idx = tid; idx < lines * NS * 32; idx += 256) {
        const int l = idx & 31, blk = idx >> 5, a = blk / NS, s = blk % NS;
        const int lg = l >> 2, lq = l & 3, hh = lq & 1;
        int sel;
        float4 v;
        v.x = sp_a_value(p.w, R, p.cf, p.cs, a, s, lg, lq, &sel);
        v.y = sp_a_value(p.w, R, p.cf, p.cs, a, s, lg + 8, lq, &sel);
        v.z = sp_a_value(p.w, R, p.cf, p.cs, a, s, lg, lq + 4, &sel);
        v.w = sp_a_value(p.w, R, p.cf, p.cs, a, s, lg + 8, lq + 4, &sel);
        uint32_t e = 0;
        for (int i = 0; i < 4; i++) {
            int s0, s1;
            sp_a_value(p.w, R, p.cf, p.cs, a, s, lg, 4 * hh + i, &s0);
            sp_a_value(p.w, R, p.cf, p.cs, a, s, lg + 8, 4 * hh + i, &s1);
            e |= (s0 ? 0xEu : 0x4u) << (4 * i);
            e |= (s1 ? 0xEu : 0x4u) << (4 * (i + 4));
        }
        Af[idx] = v;
        Em[idx] = e;
    }

    // B offsets (floats within a staged row) of this thread, for a row whose
    // chunks are not swizzled (0) and swizzled (1)
    int boff0[NS], boff1[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        const int c = 4 * ws + p.bchunk[4 * s + q];
        boff0[s] = 4 * c;
        boff1[s] = 4 * (c ^ p.sigma);
    }
    const int H = kSpTY + 2 * R, RL = p.rl, RP = 4 * PQ;
    const int64_t ny = p.Ey - 2 * p.rh, nx = p.Ex - 2 * p.rh, Ex = p.Ex;
    const size_t tile_floats = (size_t)H * RP;
    const bool dbl = p.nbuf == 2;

    // Each thread copies (and later rounds) the same elements of every tile:
    // rows warp + 8i and, in 16-byte mode, 16-byte chunks lane + 32k, else
    // columns lane + 32k of the staged window.
    auto stage = [&](int tile, float *buf) {
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int64_t Y0 = p.rh + (int64_t)ty * kSpTY - R, X0 = p.rh - p.xshift + (int64_t)tx * kSpTX - R;
        const bool inside = Y0 >= 0 && Y0 + H <= p.Ey && X0 >= 0 && X0 + RL <= Ex;
        for (int i = warp; i < H; i += 8) {
            const int sw = ((i >> 3) & 1) ? p.sigma : 0;
            const int64_t gy = Y0 + i;
            const bool rok = gy >= 0 && gy < p.Ey;
            if (p.vec16) {
                float *drow = buf + (size_t)i * RP;
                const float *srow = in + (rok ? gy : 0) * Ex;
                for (int c = lane; 4 * c < RL; c += 32) {
                    const int64_t gx = X0 + 4 * c;  // a multiple of 4: the chunk is wholly inside or outside
                    const bool ok = rok && gx >= 0 && gx < Ex;
                    cp_async16(drow + 4 * (c ^ sw), ok ? srow + gx : in, ok);
                }
                continue;
            }
            float *dst = buf + (size_t)i * RP + 4 * ((lane >> 2) ^ sw) + (lane & 3);
            if (inside) {
                const float *src = in + gy * Ex + X0 + lane;
                for (int j = 0; j + lane < RL; j += 32) cp_async4(dst + j, src + j, true);
            } else {
                for (int j = 0; j + lane < RL; j += 32) {
                    const int64_t gx = X0 + lane + j;
                    const bool ok = rok && gx >= 0 && gx < Ex;
                    cp_async4(dst + j, ok ? in + gy * Ex + gx : in, ok);
                }
            }
        }
    };
    auto round_own = [&](float *buf) {
        for (int i = warp; i < H; i += 8) {
            const int sw = ((i >> 3) & 1) ? p.sigma : 0;
            if (p.vec16) {
                float *drow = buf + (size_t)i * RP;
                for (int c = lane; 4 * c < RL; c += 32) {
                    float4 *q4 = reinterpret_cast<float4 *>(drow + 4 * (c ^ sw));
                    float4 v = *q4;
                    v.x = cvt_tf32(v.x);
                    v.y = cvt_tf32(v.y);
                    v.z = cvt_tf32(v.z);
                    v.w = cvt_tf32(v.w);
                    *q4 = v;
                }
                continue;
            }
            float *dst = buf + (size_t)i * RP + 4 * ((lane >> 2) ^ sw) + (lane & 3);
            for (int j = 0; j + lane < RL; j += 32) dst[j] = cvt_tf32(dst[j]);
        }
    };

    int cur = 0;
    if (dbl && (int)blockIdx.x < ntiles) stage(blockIdx.x, S);
    cp_async_commit();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int64_t Y0 = p.rh + (int64_t)ty * kSpTY, X0 = p.rh - p.xshift + (int64_t)tx * kSpTX;
        float *T = S + cur * tile_floats;
        if (dbl) {
            const int nxt = tile + gridDim.x;
            if (nxt < ntiles) stage(nxt, S + (cur ^ 1) * tile_floats);
            cp_async_commit();
            cp_async_wait1();  // this tile's copies have landed (the newest group may still be in flight)
        } else {
            stage(tile, T);
            cp_async_commit();
            cp_async_wait0();
        }
        round_own(T);
        __syncthreads();

        float acc[8][4];
#pragma unroll
        for (int y = 0; y < 8; y++) acc[y][0] = acc[y][1] = acc[y][2] = acc[y][3] = 0.0f;

        const float *Tw = T + (size_t)(64 * wb + 8 * g) * RP;
        int a_lo = 0;
        for (; a_lo + LC <= lines; a_lo += LC)
            sp_pass<NS, LC, FULL>(acc, Tw, a_lo, RP, boff0, boff1, g, Af, Em, p.mask, lane);
        switch (lines - a_lo) {  // the last, partial pass: no predicated-off MMAs
        case 1: sp_pass<NS, 1, FULL>(acc, Tw, a_lo, RP, boff0, boff1, g, Af, Em, p.mask, lane); break;
        case 2: if constexpr (LC > 2) sp_pass<NS, 2, FULL>(acc, Tw, a_lo, RP, boff0, boff1, g, Af, Em, p.mask, lane); break;
        case 3: if constexpr (LC > 3) sp_pass<NS, 3, FULL>(acc, Tw, a_lo, RP, boff0, boff1, g, Af, Em, p.mask, lane); break;
        case 4: if constexpr (LC > 4) sp_pass<NS, 4, FULL>(acc, Tw, a_lo, RP, boff0, boff1, g, Af, Em, p.mask, lane); break;
        default: break;
        }

        // epilogue: d0 (col g, row slot 2q), d1 (g, 2q+1), d2 (g+8, 2q), d3 (g+8, 2q+1);
        // row slot n of accumulator y0 is output row y0 + 8n of the band
        const int64_t by = Y0 + 64 * wb, bx = X0 + 16 * ws;
        const int64_t iy0 = by - p.rh, ix0 = bx - p.rh;
        const bool full = iy0 >= p.band && ix0 >= p.band && iy0 + 64 <= ny - p.band && ix0 + 16 <= nx - p.band;
        float *ob = out + (by + 16 * q) * Ex + bx + g;
        if (full) {
#pragma unroll
            for (int y0 = 0; y0 < 8; y0++) {
                ob[y0 * Ex] = acc[y0][0];
                ob[(y0 + 8) * Ex] = acc[y0][1];
                ob[y0 * Ex + 8] = acc[y0][2];
                ob[(y0 + 8) * Ex + 8] = acc[y0][3];
            }
        } else {
#pragma unroll
            for (int y0 = 0; y0 < 8; y0++) {
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const int m = g + 8 * (h >> 1), n = 2 * q + (h & 1);
                    const int64_t iy = iy0 + y0 + 8 * n, ix = ix0 + m;
                    if (iy < ny && ix < nx && iy >= p.band && ix >= p.band && ny - 1 - iy >= p.band &&
                        nx - 1 - ix >= p.band)
                        out[(iy + p.rh) * Ex + ix + p.rh] = acc[y0][h];
                }
            }
        }
        __syncthreads();  // every read of this buffer is done before it is refilled
        if (dbl) cur ^= 1;
    }
    cp_async_wait0();
}

template <int NS, int LC, bool FULL>
stencil_status launch_ns(const SpParams &sp, const void *in, void *out, int64_t ny, int64_t nx, cudaStream_t st)
{
    const size_t table = (size_t)sp.lines * NS * 32 * 20;
    const size_t tile = (size_t)(kSpTY + 2 * sp.R) * sp.pitch_q * 16;
    // double-buffered input tiles when two CTAs still fit on an SM, else one
    // buffer (the second CTA's copies overlap this one's MMAs)
    SpParams sp2 = sp;
    sp2.nbuf = table + 2 * tile <= 112 * 1024 ? 2 : 1;
    const size_t smem = table + sp2.nbuf * tile;
    if (smem > 227 * 1024) return fail(STENCIL_ERR_UNSUPPORTED, "sparse tensor-core tile does not fit in shared memory");
    auto kern = sptc2d_sweep<NS, LC, FULL>;
    stencil_status s = ensure_smem((const void *)kern, smem);
    if (s != STENCIL_OK) return s;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    s = occupancy((const void *)kern, 256, smem, &per_sm);
    if (s != STENCIL_OK) return s;
    if (per_sm < 1) return fail(STENCIL_ERR_UNSUPPORTED, "sparse tensor-core kernel cannot be resident");
    const int64_t nty = (ny + kSpTY - 1) / kSpTY, ntx = (nx + sp.xshift + kSpTX - 1) / kSpTX, ntiles = nty * ntx;
    if (ntiles > 0x7fffffff) return fail(STENCIL_ERR_UNSUPPORTED, "too many tiles");
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)sms * per_sm);
    kern<<<grid, 256, smem, st>>>((const float *)in, (float *)out, sp2, (int)ntiles, (int)ntx);
    note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e, "sptc2d_sweep launch");
}

}  // namespace

stencil_status launch_sptc_sweep(const Plan &p, const void *in, void *out, int t, cudaStream_t st)
{
    if (p.pat.d != 2 || p.dtype != STENCIL_F32)
        return fail(STENCIL_ERR_UNSUPPORTED, "sparse tensor-core path: 2-D FP32 grids only");
    const int r = p.pat.r, R = t * r;
    if (R > 12) return fail(STENCIL_ERR_UNSUPPORTED, "sparse tensor-core path: fused radius t*r must be <= 12");
    const SpLayout L = sp_layout_2d(p.pat.shape, r, t);
    SpParams sp;
    std::memset(&sp, 0, sizeof(sp));
    const std::vector<double> wt = compose_dense(p.pat, p.w, t);
    const int lines = 2 * R + 1;
    for (int i = 0; i < lines * lines; i++) sp.w[i] = wt[i];
    for (int i = 0; i < 2 * kSpMaxNs; i++) {
        sp.cf[i] = L.cf[i];
        sp.cs[i] = L.cs[i];
    }
    for (int i = 0; i < 4 * kSpMaxNs; i++) sp.bchunk[i] = i < 4 * L.ns ? L.bchunk[i] : 0;
    for (int a = 0; a < lines; a++) sp.mask[a] = (unsigned char)L.mask[a];
    sp.R = R;
    sp.rh = r;
    sp.band = (t - 1) * r;
    sp.lines = lines;
    sp.sigma = L.sigma;
    sp.pitch_q = L.pitch_q;
    sp.rl = L.rl;
    sp.Ey = p.ext[1];
    sp.Ex = p.ext[2];
    // 16-byte staging when every stored row is a 16-byte multiple and the
    // input pointer is 16-byte aligned: the first tile then starts xshift
    // columns left of the interior (its outputs there are skipped) so that
    // each tile's staged window starts on a 16-byte boundary
    sp.vec16 = (p.ext[2] % 4 == 0) && (reinterpret_cast<uintptr_t>(in) % 16 == 0);
    sp.xshift = sp.vec16 ? (int)(((r - R) % 4 + 4) % 4) : 0;
    stencil_status s;
    bool full = true;  // every line issues every instruction (no mask tests)
    for (int a = 0; a < lines; a++) full = full && L.mask[a] == (1 << L.ns) - 1;
    switch (L.ns * 2 + (full ? 1 : 0)) {
    case 4: s = launch_ns<2, 5, false>(sp, in, out, p.dims[1], p.dims[2], st); break;
    case 5: s = launch_ns<2, 5, true>(sp, in, out, p.dims[1], p.dims[2], st); break;
    case 6: s = launch_ns<3, 4, false>(sp, in, out, p.dims[1], p.dims[2], st); break;
    case 7: s = launch_ns<3, 4, true>(sp, in, out, p.dims[1], p.dims[2], st); break;
    case 8: s = launch_ns<4, 2, false>(sp, in, out, p.dims[1], p.dims[2], st); break;
    case 9: s = launch_ns<4, 2, true>(sp, in, out, p.dims[1], p.dims[2], st); break;
    default: return fail(STENCIL_ERR_UNSUPPORTED, "sparse tensor-core path: layout");
    }
    if (s != STENCIL_OK || t == 1) return s;
    return launch_cu_band(p, in, out, t, (t - 1) * r, st);
}

}  // namespace gbs
