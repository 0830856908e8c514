// cu_kernels.cuh -- CUDA-core stencil sweeps with temporal blocking.
//
// Paper Sec. 3.2.2 (CUDA cores with temporal fusion): t steps are fused in
// one pass over the grid; the intermediate steps never leave the SM, so the
// HBM traffic per point stays one read and one write (M = 2D) while the
// arithmetic grows to t * 2K (Eq. 8).
//
// One CTA owns an output tile.  It stages the tile grown by t*r on every
// side (the dependency region of t steps) from global memory into shared
// memory, then runs the t sub-steps in shared memory (ping-pong between two
// buffers); sub-step s computes the region grown by (t - s) r.  Points that
// are not interior (the fixed halo, or outside the stored array) keep their
// value, which re-imposes the Dirichlet boundary after every sub-step.  The
// last sub-step writes straight to global memory.  FP64 (and 3-D): each
// thread computes a strip of V outputs along the slowest tile axis and reuses
// every loaded input row/plane across the strip from registers.  FP32 2-D:
// each thread walks a strip of rows for four adjacent columns and rotates
// the partial sums of the 2r+1 output rows an input row touches through
// registers (f32_substep4).
//
// Weights are kernel parameters (constant bank; FP64 kernels copy them to
// shared memory), K values in the library's lexicographic offset order.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace gbs {
namespace cu {

constexpr int kThreads = 256;

template <int SHAPE, int D, int R>
struct Taps {
    static constexpr int side = 2 * R + 1;
    static constexpr int K = SHAPE == 0 ? (D == 2 ? side * side : side * side * side) : 2 * D * R + 1;
};

// Index of offset (oz, oy, ox) in the lexicographic offset list, -1 if the
// offset is not part of the pattern.  D == 2 ignores oz.
template <int SHAPE, int D, int R>
__host__ __device__ constexpr int tap_index(int oz, int oy, int ox)
{
    if (SHAPE == 0) {
        return D == 2 ? (oy + R) * (2 * R + 1) + (ox + R)
                      : ((oz + R) * (2 * R + 1) + (oy + R)) * (2 * R + 1) + (ox + R);
    }
    const int nz = (D == 3 && oz != 0) + (oy != 0) + (ox != 0);
    if (nz > 1) return -1;
    if (D == 2) {
        if (oy < 0) return oy + R;
        if (oy == 0) return 2 * R + ox;
        return 3 * R + oy;
    }
    if (oz < 0) return oz + R;
    if (oz == 0) {
        if (oy < 0) return R + oy + R;
        if (oy == 0) return 3 * R + ox;
        return 4 * R + oy;
    }
    return 5 * R + oz;
}

template <typename T, int K>
struct Weights {
    T w[K];
};

// ---------------------------------------------------------------------------
// 2-D: tile BY x BX, strips of V rows.
// ---------------------------------------------------------------------------
// Band mode (band > 0): only the tiles of the ring of tile rows/columns that
// touch the band run (a 1-D grid, ring.count blocks), and only points closer
// than `band` to the interior boundary are written.  Used after a
// tensor-core sweep, whose fused kernel is exact only away from the
// boundary.
struct Ring {
    int band;        // 0: every tile, row-major over ntx columns
    int nty, ntx;    // tiles along y and x
    int rows_tb;     // tile rows taken whole: min(nty, top_w + bottom rows)
    int top_w;       // tile rows touching the top band
    int cols_lr;     // tile columns taken in the other rows: min(ntx, left_w + right cols)
    int left_w;      // tile columns touching the left band
    int xshift;      // band 0, FP32: the tile grid starts xshift columns further left so that
                     // every staged window begins on a 16-byte boundary (then vec16 = 1)
    int vec16;       // stage interior tiles with 16-byte copies
};

// Tile id -> (tile row, tile column): first the whole tile rows (the top_w
// top ones, then the bottom ones), then, row by row, the left and right tile
// columns of the remaining rows.
__device__ __forceinline__ void ring_tile(const Ring &g, int id, int *by, int *bx)
{
    if (id < g.rows_tb * g.ntx) {
        const int rr = id / g.ntx;
        *bx = id % g.ntx;
        *by = rr < g.top_w ? rr : g.nty - g.rows_tb + rr;
    } else {
        const int id2 = id - g.rows_tb * g.ntx;
        const int cc = id2 % g.cols_lr;
        *by = g.top_w + id2 / g.cols_lr;
        *bx = cc < g.left_w ? cc : g.ntx - g.cols_lr + cc;
    }
}

// Asynchronous global -> shared copy of one element (cp.async, L1-allocating);
// src_bytes = 0 writes zeros without reading global memory.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void *smem_dst, const void *gmem_src, bool valid)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    const int n = valid ? BYTES : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(gmem_src), "n"(BYTES), "r"(n)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// f(integral_constant<int, 0>), f(<1>), ... f(<N-1>) while f returns true:
// a loop whose index is a compile-time constant in the body.
template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (void)(f(std::integral_constant<int, I>{}) && ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// FP32 sub-step, register-rotation form.  A work item is a pair of adjacent
// columns (x, x+1) and a strip of S output rows.  The thread walks down the
// strip's input rows once; each row window is read with 8-byte shared loads
// (D = parity of the window start) and added to the 2R+1 output rows it
// touches, whose partial sums rotate through 2R+1 register slots.  The row
// loop is unrolled by 2R+1, so every slot index and weight index is a
// compile-time constant and no FMA carries a condition; output row jj is
// complete after input row jj + 2R and is stored from its slot.  When the
// whole region is interior the stores skip the boundary tests.
template <int SHAPE, int R, int D, typename WT>
__device__ __forceinline__ void f32_substep(const float *__restrict__ src, float *__restrict__ dst,
                                            float *__restrict__ out, const WT &wt, int W, int H, int lo, int hiY,
                                            int hiX, int64_t Y0, int64_t X0, int64_t Ey, int64_t Ex, bool last,
                                            bool all_interior, int band)
{
    constexpr int NS = 2 * R + 1;      // rotating slots
    constexpr int NV = 2 * R + 2 + D;  // window values per row
    constexpr int NL = (NV + 1) / 2;   // float2 loads per row
    const int cw = hiX - lo, ch = hiY - lo;
    const int npairs = (cw + 1) / 2;
    // strips of ~16 rows (the 2R extra input rows per strip are the only
    // redundant work), enough of them to give every thread work
    const int nstrips = max(1, min((ch + 15) / 16, (int)((blockDim.x + npairs - 1) / npairs)));
    const int S = (ch + nstrips - 1) / nstrips;
    const int64_t ny = Ey - 2 * R, nx = Ex - 2 * R;

    const bool fast = all_interior && band == 0;
    auto store = [&](int y, int x, float v0, float v1, bool second) {
        if (fast) {
            if (last) {
                float *o = out + (Y0 + y) * Ex + (X0 + x);
                if (second && ((reinterpret_cast<uintptr_t>(o) & 7) == 0)) {
                    *reinterpret_cast<float2 *>(o) = make_float2(v0, v1);
                } else {
                    o[0] = v0;
                    if (second) o[1] = v1;
                }
            } else {
                // W is even, so dst + y*W + x is 8-byte aligned exactly when x is
                // even (x has the parity of s*R: uniform over the sub-step)
                float *o = dst + y * W + x;
                if (second && (x & 1) == 0) {
                    *reinterpret_cast<float2 *>(o) = make_float2(v0, v1);
                } else {
                    o[0] = v0;
                    if (second) o[1] = v1;
                }
            }
            return;
        }
        const int64_t gy = Y0 + y, gx = X0 + x;
        const bool rowint = gy >= R && gy < Ey - R;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !second) break;
            const int64_t gxh = gx + h;
            const bool interior = rowint && gxh >= R && gxh < Ex - R;
            const float val = h ? v1 : v0;
            if (last) {
                bool keep = interior;
                if (band > 0) {
                    const int64_t iy = gy - R, ix = gxh - R;
                    keep = keep && (iy < band || ix < band || ny - 1 - iy < band || nx - 1 - ix < band);
                }
                if (keep) out[gy * Ex + gxh] = val;
            } else {
                dst[y * W + x + h] = interior ? val : src[y * W + x + h];
            }
        }
    };

    for (int item = threadIdx.x; item < nstrips * npairs; item += blockDim.x) {
        const int sy = item / npairs, px = item - sy * npairs;
        const int y0 = lo + sy * S;
        const int yend = min(y0 + S, hiY);  // outputs y0 .. yend-1
        if (y0 >= yend) continue;
        const int x = lo + 2 * px;
        const bool second = x + 1 < hiX;
        const int nrows = (yend - y0) + 2 * R;  // input rows y0-R .. yend-1+R
        float a0[NS], a1[NS];
#pragma unroll
        for (int m = 0; m < NS; ++m) a0[m] = a1[m] = 0.0f;
        const float *col = src + x - R - D;
        for (int base = 0; base < nrows; base += NS) {
#pragma unroll
            for (int u = 0; u < NS; ++u) {
                const int qq = base + u;  // relative input row; absolute row y0 - R + qq
                if (qq < nrows) {
                    const float2 *row = reinterpret_cast<const float2 *>(col + (y0 - R + qq) * W);
                    float v[2 * NL];
#pragma unroll
                    for (int c = 0; c < NL; ++c) {
                        const float2 t2 = row[c];
                        v[2 * c] = t2.x;
                        v[2 * c + 1] = t2.y;
                    }
                    // output jj = qq - e (e = 0..2R) takes this row with oy = e - R
#pragma unroll
                    for (int e = 0; e < NS; ++e) {
                        const int slot = ((u - e) % NS + NS) % NS;
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            const int k = tap_index<SHAPE, 2, R>(0, e - R, ox);
                            if (k >= 0) {
                                a0[slot] = fmaf(wt.w[k], v[D + R + ox], a0[slot]);
                                a1[slot] = fmaf(wt.w[k], v[D + R + ox + 1], a1[slot]);
                            }
                        }
                    }
                    // output jj = qq - 2R is complete (slot (u - 2R) mod NS = (u + 1) mod NS)
                    constexpr int dummy = 0;
                    (void)dummy;
                    const int jj = qq - 2 * R;
                    const int done = (u + 1) % NS;
                    if (jj >= 0) store(y0 + jj, x, a0[done], a1[done], second);
                    a0[done] = 0.0f;
                    a1[done] = 0.0f;
                }
            }
        }
    }
}

// Row pitch of a staged tile row of width W and the elements of one staging
// buffer of H rows: FP32 rows are padded to 16-byte multiples (the 4-column
// sub-step reads them with 16-byte loads) and each buffer has 8 elements of
// slack at its end (the last window of the last row reads past column W).
template <typename T>
__host__ __device__ constexpr int row_pitch(int W)
{
    return sizeof(T) == 4 ? (W + 3) & ~3 : W;
}
template <typename T>
__host__ __device__ constexpr size_t buf_elems(int H, int W)
{
    return (size_t)H * row_pitch<T>(W) + (sizeof(T) == 4 ? 8 : 0);
}

// FP32 sub-step, 4-column register-rotation form.  A work item is a quad of
// adjacent columns (x .. x+3) and a strip of S output rows.  The thread walks
// down the strip's input rows once; each row window (columns x-R-D ..,
// D = (lo-R) mod 4 so the window starts on a 16-byte boundary) is read with
// 16-byte shared loads and added to the 2R+1 output rows it touches, whose
// partial sums rotate through 2R+1 register slots.  The first 2R+1 input rows
// are peeled so that no FMA goes into an output above the strip; the row loop
// is unrolled by 2R+1, so every slot and weight index is a compile-time
// constant.  Output row jj is complete after input row jj + 2R and is stored
// (as two 8-byte or four 4-byte stores, by alignment) from its slot.  P is
// the row pitch of src and dst (a multiple of 4).
template <int SHAPE, int R, int D, typename WT>
__device__ __forceinline__ void f32_substep4(const float *__restrict__ src, float *__restrict__ dst,
                                             float *__restrict__ out, const WT &wt, int P, int lo, int hiY, int hiX,
                                             int64_t Y0, int64_t X0, int64_t Ey, int64_t Ex, bool last,
                                             bool all_interior, int band)
{
    constexpr int NS = 2 * R + 1;          // rotating slots
    constexpr int NV = 2 * R + 4 + D;      // window values per row
    constexpr int NL = (NV + 3) / 4;       // 16-byte loads per row
    const int cw = hiX - lo, ch = hiY - lo;
    const int nquads = (cw + 3) / 4;
    // enough strips to give every thread a work item, each of >= 4 rows
    const int nstrips = max(1, min(max(1, ch / 4), (int)((blockDim.x + nquads - 1) / nquads)));
    const int S = (ch + nstrips - 1) / nstrips;
    const int64_t ny = Ey - 2 * R, nx = Ex - 2 * R;
    const bool fast = all_interior && band == 0;

    for (int item = threadIdx.x; item < nstrips * nquads; item += blockDim.x) {
        const int sy = item / nquads, qx = item - sy * nquads;
        const int y0 = lo + sy * S;
        const int yend = min(y0 + S, hiY);  // outputs y0 .. yend-1
        if (y0 >= yend) continue;
        const int x = lo + 4 * qx;
        const int nval = min(4, hiX - x);
        const int nrows = (yend - y0) + 2 * R;  // input rows y0-R .. yend-1+R
        const float *col = src + x - R - D;
        // output store of row y (4 values), by alignment and boundary
        auto store = [&](int y, const float (&a)[4]) {
            if (fast && nval == 4) {
                float *o = last ? out + (Y0 + y) * Ex + (X0 + x) : dst + y * P + x;
                const uintptr_t al = reinterpret_cast<uintptr_t>(o) & 15;
                if (al == 0) {
                    *reinterpret_cast<float4 *>(o) = make_float4(a[0], a[1], a[2], a[3]);
                } else if ((al & 7) == 0) {
                    reinterpret_cast<float2 *>(o)[0] = make_float2(a[0], a[1]);
                    reinterpret_cast<float2 *>(o)[1] = make_float2(a[2], a[3]);
                } else {
                    o[0] = a[0];
                    o[1] = a[1];
                    o[2] = a[2];
                    o[3] = a[3];
                }
                return;
            }
            const int64_t gy = Y0 + y;
            const bool rowint = gy >= R && gy < Ey - R;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                if (h >= nval) break;
                const int64_t gx = X0 + x + h;
                const bool interior = rowint && gx >= R && gx < Ex - R;
                if (last) {
                    bool keep = interior;
                    if (band > 0) {
                        const int64_t iy = gy - R, ix = gx - R;
                        keep = keep && (iy < band || ix < band || ny - 1 - iy < band || nx - 1 - ix < band);
                    }
                    if (keep) out[gy * Ex + gx] = a[h];
                } else {
                    dst[y * P + x + h] = interior ? a[h] : src[y * P + x + h];
                }
            }
        };
        float acc[NS][4];
#pragma unroll
        for (int m = 0; m < NS; ++m) acc[m][0] = acc[m][1] = acc[m][2] = acc[m][3] = 0.0f;
        // one input row (relative row qq, unrolled position u) into the slots
        // of outputs qq - e for e in [0, e_hi]
        auto row = [&](int qq, int u, int e_hi) {
            const float4 *rp = reinterpret_cast<const float4 *>(col + (y0 - R + qq) * P);
            float v[4 * NL];
#pragma unroll
            for (int c = 0; c < NL; ++c) {
                const float4 t4 = rp[c];
                v[4 * c] = t4.x;
                v[4 * c + 1] = t4.y;
                v[4 * c + 2] = t4.z;
                v[4 * c + 3] = t4.w;
            }
#pragma unroll
            for (int e = 0; e < NS; ++e) {
                if (e > e_hi) continue;
                const int slot = ((u - e) % NS + NS) % NS;
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    const int k = tap_index<SHAPE, 2, R>(0, e - R, ox);
                    if (k >= 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[slot][c] = fmaf(wt.w[k], v[D + R + ox + c], acc[slot][c]);
                    }
                }
            }
        };
        // head: input row u (u <= 2R) feeds only outputs u - e >= 0
#pragma unroll
        for (int u = 0; u < NS; ++u)
            if (u < nrows) row(u, u, u);
        if (2 * R < nrows) {  // output 0 is complete after row 2R (slot 0)
            store(y0, acc[0]);
            acc[0][0] = acc[0][1] = acc[0][2] = acc[0][3] = 0.0f;
        }
        for (int base = NS; base < nrows; base += NS) {
#pragma unroll
            for (int u = 0; u < NS; ++u) {
                const int qq = base + u;
                if (qq < nrows) {
                    row(qq, u, 2 * R);
                    const int jj = qq - 2 * R;  // complete output
                    const int done = (u + 1) % NS;
                    store(y0 + jj, acc[done]);
                    acc[done][0] = acc[done][1] = acc[done][2] = acc[done][3] = 0.0f;
                }
            }
        }
    }
}

// FP32 sub-step, fixed-strip form: the fast case of f32_substep4 (every point
// of the region interior, no band, whole quads: cw a multiple of 4,
// ch >= S).  A work item is a quad of columns and S output rows, S a
// compile-time constant: the S + 2R input rows are unrolled completely, so
// each input row goes exactly into the outputs it touches (no partial sums
// of rows outside the strip, no slot rotation) and every index is a
// constant.  When ch is not a multiple of S the last strip of a column
// starts at hiY - S and overlaps the one above; the overlapping outputs are
// computed twice with identical values.  Stores are 16- or 8-byte vectors
// (the alignment of x0 + x is the same for every item of the sub-step).
template <int SHAPE, int R, int D, int S, typename WT>
__device__ __forceinline__ void f32_substep4_fixed(const float *__restrict__ src, float *__restrict__ dst,
                                                   float *__restrict__ out, const WT &wt, int P, int lo, int hiY,
                                                   int hiX, int64_t Y0, int64_t X0, int64_t Ex, bool last)
{
    constexpr int NV = 2 * R + 4 + D;  // window values per row
    constexpr int NL = (NV + 3) / 4;   // 16-byte loads per row
    constexpr int NR = S + 2 * R;      // input rows per strip
    const int nquads = (hiX - lo) >> 2;
    const int nstrips = (hiY - lo + S - 1) / S;
    const int nitems = nquads * nstrips;
    // outputs: (row y, column x) of the region is obase[off0 + y * pitch + x]
    float *const obase = last ? out : dst;
    const int64_t off0 = last ? Y0 * Ex + X0 : 0;
    const int64_t pitch = last ? Ex : P;
    // element offset of the first output within its 16-byte chunk: the same
    // for every item when the pitch is a multiple of 4 (else scalar stores)
    const int phase = (pitch & 3) ? 1
                                  : (int)(((reinterpret_cast<uintptr_t>(obase) >> 2) +
                                           (uint64_t)(off0 + (int64_t)lo * pitch + lo)) & 3);
    for (int item = threadIdx.x; item < nitems; item += blockDim.x) {
        const int sy = item / nquads, qx = item - sy * nquads;
        const int y0 = min(lo + sy * S, hiY - S);
        const int x = lo + 4 * qx;
        const float4 *rp = reinterpret_cast<const float4 *>(src + (y0 - R) * P + x - R - D);
        const int p4 = P >> 2;
        float acc[S][4];
#pragma unroll
        for (int j = 0; j < S; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            float v[4 * NL];
#pragma unroll
            for (int c = 0; c < NL; ++c) {
                const float4 t4 = rp[q * p4 + c];
                v[4 * c] = t4.x;
                v[4 * c + 1] = t4.y;
                v[4 * c + 2] = t4.z;
                v[4 * c + 3] = t4.w;
            }
            // input row q (row y0 - R + q) feeds outputs j = q - R - oy, oy in [-R, R]
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const int oy = q - R - j;
                if (oy < -R || oy > R) continue;
#pragma unroll
                for (int ox = -R; ox <= R; ++ox) {
                    const int k = tap_index<SHAPE, 2, R>(0, oy, ox);
                    if (k >= 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[j][c] = fmaf(wt.w[k], v[D + R + ox + c], acc[j][c]);
                    }
                }
            }
        }
        float *o = obase + (off0 + (int64_t)y0 * pitch + x);
        if (phase == 0) {
#pragma unroll
            for (int j = 0; j < S; ++j)
                *reinterpret_cast<float4 *>(o + j * pitch) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        } else if (phase == 2) {
#pragma unroll
            for (int j = 0; j < S; ++j) {
                float2 *o2 = reinterpret_cast<float2 *>(o + j * pitch);
                o2[0] = make_float2(acc[j][0], acc[j][1]);
                o2[1] = make_float2(acc[j][2], acc[j][3]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < S; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) o[j * pitch + c] = acc[j][c];
        }
    }
}

// Selects the window phase D = (lo - R) mod 4 and the strip height (4 or 8)
// of f32_substep4_fixed.
template <int SHAPE, int R, typename WT>
__device__ __forceinline__ void f32_fixed_dispatch(int D, bool s4, const float *__restrict__ src,
                                                   float *__restrict__ dst, float *__restrict__ out, const WT &wt,
                                                   int P, int lo, int hiY, int hiX, int64_t Y0, int64_t X0,
                                                   int64_t Ex, bool last)
{
#define GBS_FIXED(DD)                                                                                          \
    if (s4)                                                                                                    \
        f32_substep4_fixed<SHAPE, R, DD, 4>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last);             \
    else                                                                                                       \
        f32_substep4_fixed<SHAPE, R, DD, 8>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last);
    switch (D) {
    case 0: GBS_FIXED(0) break;
    case 1: GBS_FIXED(1) break;
    case 2: GBS_FIXED(2) break;
    default: GBS_FIXED(3) break;
    }
#undef GBS_FIXED
}

// f32_substep4_fixed with strips of 2 rows (radii 3 and more).
template <int SHAPE, int R, typename WT>
__device__ __forceinline__ void f32_fixed_dispatch2(int D, const float *__restrict__ src, float *__restrict__ dst,
                                                    float *__restrict__ out, const WT &wt, int P, int lo, int hiY,
                                                    int hiX, int64_t Y0, int64_t X0, int64_t Ex, bool last)
{
    switch (D) {
    case 0: f32_substep4_fixed<SHAPE, R, 0, 2>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last); break;
    case 1: f32_substep4_fixed<SHAPE, R, 1, 2>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last); break;
    case 2: f32_substep4_fixed<SHAPE, R, 2, 2>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last); break;
    default: f32_substep4_fixed<SHAPE, R, 3, 2>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex, last); break;
    }
}

// Persistent form: CTA b processes tiles b, b + gridDim.x, ...; while it
// computes one tile it prefetches the next into the other staging buffer
// with cp.async, so the FMA pipe never waits for a synchronous load phase.
// Shared memory: two staging buffers (H x W) and, for t > 1, a work buffer
// for the intermediate sub-steps.
// FP64 kernels read their weights from shared memory (one LDS per FMA is
// free next to the FP64 pipe, and keeping K doubles in registers across the
// persistent loop would spill); FP32 kernels read them from the constant bank.
template <typename T, int K>
__host__ __device__ constexpr int weight_smem_bytes()
{
    return sizeof(T) == 8 ? (int)((K * sizeof(T) + 15) / 16 * 16) : 0;
}

template <typename T, int SHAPE, int R, int V>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && R <= 3) ? 3 : 2)
    cu2d_sweep(const T *__restrict__ in, T *__restrict__ out,
               const __grid_constant__ Weights<T, Taps<SHAPE, 2, R>::K> wt, int64_t Ey, int64_t Ex, int BY, int BX,
               int t, const Ring ring, int ntiles)
{
    constexpr int KT = Taps<SHAPE, 2, R>::K;
    constexpr bool kSmemW = sizeof(T) == 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *wsm = reinterpret_cast<T *>(smem_raw);
    if (kSmemW) {
        for (int k = threadIdx.x; k < KT; k += blockDim.x) wsm[k] = wt.w[k];
    }
    unsigned char *base = smem_raw + weight_smem_bytes<T, KT>();
    const int H = BY + 2 * t * R, W = BX + 2 * t * R, P = row_pitch<T>(W);
    const size_t buf = buf_elems<T>(H, W);
    T *const stage0 = reinterpret_cast<T *>(base), *const stage1 = stage0 + buf;
    T *work = reinterpret_cast<T *>(base) + 2 * buf;
    const int64_t ny = Ey - 2 * R, nx = Ex - 2 * R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    auto origin = [&](int id, int64_t *Y0, int64_t *X0) {
        int by, bx;
        if (ring.band > 0) {
            ring_tile(ring, id, &by, &bx);
        } else {
            by = id / ring.ntx;
            bx = id % ring.ntx;
        }
        *Y0 = R + (int64_t)by * BY - (int64_t)t * R;
        *X0 = R + (int64_t)bx * BX - (int64_t)t * R - ring.xshift;
    };
    // Stage the dependency region of a tile; cells outside the stored array
    // are zero-filled and never used by an interior point.
    auto prefetch = [&](int id, T *dst) {
        int64_t Y0, X0;
        origin(id, &Y0, &X0);
        if (sizeof(T) == 4 && ring.vec16 && Y0 >= 0 && X0 >= 0 && Y0 + H <= Ey && X0 + P <= Ex) {
            // 16-byte copies: X0, the row length and the input are 16-byte aligned
            const T *g = in + Y0 * Ex + X0;
            for (int y = warp; y < H; y += nwarps) {
                const T *grow = g + y * Ex;
                T *srow = dst + y * P;
                for (int c = lane; 4 * c < W; c += 32) cp_async_elem<16>(srow + 4 * c, grow + 4 * c, true);
            }
            return;
        }
        if (Y0 >= 0 && X0 >= 0 && Y0 + H <= Ey && X0 + W <= Ex) {
            // the whole region lies in the stored array: no per-element tests
            const T *g = in + Y0 * Ex + X0;
            for (int y = warp; y < H; y += nwarps) {
                const T *grow = g + y * Ex;
                T *srow = dst + y * P;
                for (int x = lane; x < W; x += 32) cp_async_elem<sizeof(T)>(srow + x, grow + x, true);
            }
            return;
        }
        for (int y = warp; y < H; y += nwarps) {
            const int64_t gy = Y0 + y;
            const bool rowok = gy >= 0 && gy < Ey;
            for (int x = lane; x < W; x += 32) {
                const int64_t gx = X0 + x;
                const bool ok = rowok && gx >= 0 && gx < Ex;
                cp_async_elem<sizeof(T)>(dst + y * P + x, ok ? in + gy * Ex + gx : in, ok);
            }
        }
    };

    int cur = 0;
    if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x, stage0);
    cp_async_commit();
    for (int id = blockIdx.x; id < ntiles; id += gridDim.x) {
        const int nid = id + gridDim.x;
        if (nid < ntiles) prefetch(nid, cur ? stage0 : stage1);
        cp_async_commit();
        cp_async_wait_group<1>();  // this tile's copies (all but the newest group) have landed
        __syncthreads();
        int64_t Y0, X0;
        origin(id, &Y0, &X0);

        T *src = cur ? stage1 : stage0, *dst = work;
        for (int s = 1; s <= t; ++s) {
            const int lo = s * R;
            const int hiY = H - s * R, hiX = W - s * R;
            const int cw = hiX - lo, ch = hiY - lo;
            const int strips = (ch + V - 1) / V;
            const bool last = s == t;
            if constexpr (sizeof(T) == 4) {
                const bool all_int = Y0 + lo >= R && Y0 + hiY <= Ey - R && X0 + lo >= R && X0 + hiX <= Ex - R;
                if constexpr (R <= 2) {
                    if (all_int && ring.band == 0 && (cw & 3) == 0 && ch >= 8) {
                        // strips of 8 rows, or of 4 when that tiles the region exactly
                        const bool s4 = (ch & 7) != 0 && (ch & 3) == 0;
                        f32_fixed_dispatch<SHAPE, R>((lo - R) & 3, s4, src, dst, out, wt, P, lo, hiY, hiX, Y0, X0,
                                                     Ex, last);
                        __syncthreads();
                        T *tmp = src;
                        src = dst;
                        dst = tmp;
                        continue;
                    }
                } else {
                    // larger radii: strips of 2 rows (each item reads 2 + 2R rows
                    // for 8 outputs: loads stay a few % of the (2R+1)^2 taps, and
                    // the unrolled code stays a few thousand FMAs)
                    if (all_int && ring.band == 0 && (cw & 3) == 0 && ch >= 2) {
                        f32_fixed_dispatch2<SHAPE, R>((lo - R) & 3, src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ex,
                                                      last);
                        __syncthreads();
                        T *tmp = src;
                        src = dst;
                        dst = tmp;
                        continue;
                    }
                }
                switch ((lo - R) & 3) {  // offset of the first window within its 16-byte chunk
                case 0:
                    f32_substep4<SHAPE, R, 0>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ey, Ex, last, all_int,
                                              ring.band);
                    break;
                case 1:
                    f32_substep4<SHAPE, R, 1>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ey, Ex, last, all_int,
                                              ring.band);
                    break;
                case 2:
                    f32_substep4<SHAPE, R, 2>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ey, Ex, last, all_int,
                                              ring.band);
                    break;
                default:
                    f32_substep4<SHAPE, R, 3>(src, dst, out, wt, P, lo, hiY, hiX, Y0, X0, Ey, Ex, last, all_int,
                                              ring.band);
                    break;
                }
                __syncthreads();
                T *tmp = src;
                src = dst;
                dst = tmp;
                continue;
            }
            for (int item = threadIdx.x; item < cw * strips; item += blockDim.x) {
                const int x = lo + item % cw;
                const int y0 = lo + (item / cw) * V;
                T acc[V];
#pragma unroll
                for (int j = 0; j < V; ++j) acc[j] = T(0);
#pragma unroll
                for (int q = 0; q < V + 2 * R; ++q) {
                    const int yy = y0 - R + q;
                    if (yy < H) {
                        const T *row = src + yy * P + x;
                        T v[2 * R + 1];
#pragma unroll
                        for (int c = 0; c < 2 * R + 1; ++c) v[c] = row[c - R];
#pragma unroll
                        for (int j = 0; j < V; ++j) {
                            const int oy = q - R - j;
                            if (oy >= -R && oy <= R) {
#pragma unroll
                                for (int ox = -R; ox <= R; ++ox) {
                                    const int k = tap_index<SHAPE, 2, R>(0, oy, ox);
                                    if (k >= 0) acc[j] = fma(kSmemW ? wsm[k] : wt.w[k], v[ox + R], acc[j]);
                                }
                            }
                        }
                    }
                }
                const int64_t gx = X0 + x;
                const bool colint = gx >= R && gx < Ex - R;
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int y = y0 + j;
                    if (y < hiY) {
                        const int64_t gy = Y0 + y;
                        const bool interior = colint && gy >= R && gy < Ey - R;
                        if (last) {
                            bool keep = interior;
                            if (ring.band > 0) {
                                const int64_t iy = gy - R, ix = gx - R;
                                keep = keep && (iy < ring.band || ix < ring.band || ny - 1 - iy < ring.band ||
                                                nx - 1 - ix < ring.band);
                            }
                            if (keep) out[gy * Ex + gx] = acc[j];
                        } else {
                            dst[y * P + x] = interior ? acc[j] : src[y * P + x];
                        }
                    }
                }
            }
            __syncthreads();
            // next sub-step reads what this one wrote; the staged input is no
            // longer needed after the first sub-step, so it becomes the target
            T *tmp = src;
            src = dst;
            dst = tmp;
        }
        cur ^= 1;
    }
    cp_async_wait_group<0>();
}

// ---------------------------------------------------------------------------
// 3-D: tile BZ x BY x BX, strips of V planes.
// ---------------------------------------------------------------------------
template <typename T, int SHAPE, int R, int V>
__global__ void __launch_bounds__(kThreads, 2)
    cu3d_sweep(const T *__restrict__ in, T *__restrict__ out,
               const __grid_constant__ Weights<T, Taps<SHAPE, 3, R>::K> wt, int64_t Ez, int64_t Ey, int64_t Ex,
               int BZ, int BY, int BX, int t, int tiles_x, int tiles_y, int ntiles)
{
    constexpr int KT = Taps<SHAPE, 3, R>::K;
    constexpr bool kSmemW = sizeof(T) == 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *wsm = reinterpret_cast<T *>(smem_raw);
    if (kSmemW) {
        for (int k = threadIdx.x; k < KT; k += blockDim.x) wsm[k] = wt.w[k];
    }
    unsigned char *base = smem_raw + weight_smem_bytes<T, KT>();
    const int Z = BZ + 2 * t * R, H = BY + 2 * t * R, W = BX + 2 * t * R;
    const int plane = H * W;
    const size_t buf = (size_t)Z * plane;
    T *stage[2] = {reinterpret_cast<T *>(base), reinterpret_cast<T *>(base) + buf};
    T *work = reinterpret_cast<T *>(base) + 2 * buf;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

    auto origin = [&](int id, int64_t *Z0, int64_t *Y0, int64_t *X0) {
        const int bx = id % tiles_x, by = (id / tiles_x) % tiles_y, bz = id / (tiles_x * tiles_y);
        *Z0 = R + (int64_t)bz * BZ - (int64_t)t * R;
        *Y0 = R + (int64_t)by * BY - (int64_t)t * R;
        *X0 = R + (int64_t)bx * BX - (int64_t)t * R;
    };
    auto prefetch = [&](int id, T *dst) {
        int64_t Z0, Y0, X0;
        origin(id, &Z0, &Y0, &X0);
        for (int zy = warp; zy < Z * H; zy += nwarps) {
            const int z = zy / H, y = zy % H;
            const int64_t gz = Z0 + z, gy = Y0 + y;
            const bool ok = gz >= 0 && gz < Ez && gy >= 0 && gy < Ey;
            const T *row = in + (gz * Ey + gy) * Ex;
            for (int x = lane; x < W; x += 32) {
                const int64_t gx = X0 + x;
                const bool v = ok && gx >= 0 && gx < Ex;
                cp_async_elem<sizeof(T)>(dst + z * plane + y * W + x, v ? row + gx : in, v);
            }
        }
    };

    int cur = 0;
    if ((int)blockIdx.x < ntiles) prefetch(blockIdx.x, stage[0]);
    cp_async_commit();
    for (int id = blockIdx.x; id < ntiles; id += gridDim.x) {
        const int nid = id + gridDim.x;
        if (nid < ntiles) prefetch(nid, stage[cur ^ 1]);
        cp_async_commit();
        cp_async_wait_group<1>();
        __syncthreads();
        int64_t Z0, Y0, X0;
        origin(id, &Z0, &Y0, &X0);

        T *src = stage[cur], *dst = work;
        for (int s = 1; s <= t; ++s) {
            const int lo = s * R;
            const int hiZ = Z - s * R, hiY = H - s * R, hiX = W - s * R;
            const int cw = hiX - lo, ch = hiY - lo, cz = hiZ - lo;
            const int strips = (cz + V - 1) / V;
            const bool last = s == t;
            for (int item = threadIdx.x; item < cw * ch * strips; item += blockDim.x) {
                const int x = lo + item % cw;
                const int y = lo + (item / cw) % ch;
                const int z0 = lo + (item / (cw * ch)) * V;
                T acc[V];
#pragma unroll
                for (int j = 0; j < V; ++j) acc[j] = T(0);
#pragma unroll
                for (int q = 0; q < V + 2 * R; ++q) {
                    const int zz = z0 - R + q;
                    if (zz < Z) {
                        const T *pl = src + zz * plane + y * W + x;
#pragma unroll
                        for (int j = 0; j < V; ++j) {
                            const int oz = q - R - j;
                            if (oz >= -R && oz <= R) {
#pragma unroll
                                for (int oy = -R; oy <= R; ++oy) {
#pragma unroll
                                    for (int ox = -R; ox <= R; ++ox) {
                                        const int k = tap_index<SHAPE, 3, R>(oz, oy, ox);
                                        if (k >= 0)
                                            acc[j] = fma(kSmemW ? wsm[k] : wt.w[k], pl[oy * W + ox], acc[j]);
                                    }
                                }
                            }
                        }
                    }
                }
                const int64_t gx = X0 + x, gy = Y0 + y;
                const bool lineint = gx >= R && gx < Ex - R && gy >= R && gy < Ey - R;
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int z = z0 + j;
                    if (z < hiZ) {
                        const int64_t gz = Z0 + z;
                        const bool interior = lineint && gz >= R && gz < Ez - R;
                        if (last) {
                            if (interior) out[(gz * Ey + gy) * Ex + gx] = acc[j];
                        } else {
                            const int o = z * plane + y * W + x;
                            dst[o] = interior ? acc[j] : src[o];
                        }
                    }
                }
            }
            __syncthreads();
            T *tmp = src;
            src = dst;
            dst = tmp;
        }
        cur ^= 1;
    }
    cp_async_wait_group<0>();
}

// ---------------------------------------------------------------------------
// 3-D, one step per sweep (t = 1), 2.5-D streaming: a work item is a
// (BY x BX) tile of one z chunk of CZ planes.  The CTA marches along z with a
// ring of NP = 2R + 1 + PF input planes (each the tile grown by R in y and x)
// in shared memory: while plane z is computed, planes z + R + 1 ..
// z + R + PF are in flight (cp.async, 16-byte copies where the stored rows
// allow), so every input plane is read once per tile and the only re-reads
// are the y/x halo.  256 threads: thread (ty, tx) = (tid / 16, tid % 16)
// computes outputs (y, x0 .. x0 + 3) for x0 = 4 tx and the RPT rows
// y = ty + 16 i; each (oz, oy) row segment of 4 + 2R values is read with
// 16-byte shared loads (rows padded to 16 bytes) and used for the 4 outputs.
// ---------------------------------------------------------------------------
constexpr int kStreamCZ = 64;

template <typename T>
__host__ __device__ constexpr int stream_rows_per_thread()
{
    return sizeof(T) == 4 ? 2 : 1;  // BY = 16 * RPT: 32 (FP32), 16 (FP64)
}

// Staged row pitch: BX = 64 plus the x halo, padded to 16 bytes.
template <typename T, int R>
__host__ __device__ constexpr int stream_pitch()
{
    return (64 + 2 * R + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T));
}

template <typename T, int R>
__host__ __device__ constexpr int stream_plane_elems()
{
    return (16 * stream_rows_per_thread<T>() + 2 * R) * stream_pitch<T, R>();
}

// Planes in flight ahead of the computed one: as many as fit (up to 4) in
// ~110 KB of ring, so that two CTAs share an SM.
template <typename T, int R>
__host__ __device__ constexpr int stream_prefetch()
{
    return (110 * 1024 / (stream_plane_elems<T, R>() * (int)sizeof(T)) - (2 * R + 1)) > 4
               ? 4
               : ((110 * 1024 / (stream_plane_elems<T, R>() * (int)sizeof(T)) - (2 * R + 1)) < 1
                      ? 1
                      : (110 * 1024 / (stream_plane_elems<T, R>() * (int)sizeof(T)) - (2 * R + 1)));
}

template <typename T, int R>
__host__ __device__ constexpr size_t stream_smem_bytes(int K)
{
    return (sizeof(T) == 8 ? (size_t)((K * sizeof(T) + 15) / 16 * 16) : 0) +
           (size_t)(2 * R + 1 + stream_prefetch<T, R>()) * stream_plane_elems<T, R>() * sizeof(T);
}

// Columns [lo, hi] of a thread's row segment (of 4 + 2R values) that the
// taps of plane offset oz, row offset oy touch: x0 + R + ox + c for the ox
// with a tap and c = 0..3 (lo > hi: no tap in this row).
template <int SHAPE, int R>
__host__ __device__ constexpr int seg_lo(int oz, int oy)
{
    int lo = 1 << 20;
    for (int ox = -R; ox <= R; ++ox)
        if (tap_index<SHAPE, 3, R>(oz, oy, ox) >= 0 && R + ox < lo) lo = R + ox;
    return lo;
}
template <int SHAPE, int R>
__host__ __device__ constexpr int seg_hi(int oz, int oy)
{
    int hi = -1;
    for (int ox = -R; ox <= R; ++ox)
        if (tap_index<SHAPE, 3, R>(oz, oy, ox) >= 0 && R + ox + 3 > hi) hi = R + ox + 3;
    return hi;
}

// v[i] = rowp[i] for i in [lo, hi] with the widest shared loads their
// alignment allows (rowp is 16-byte aligned): 16-byte, then 8-byte (FP32),
// then single loads.  lo and hi are constants once the callers' loops over
// the tap offsets are unrolled, so every branch folds away.
template <typename T, int NV>
__device__ __forceinline__ void load_seg(const T *__restrict__ rowp, T *v, int lo, int hi)
{
    constexpr int VE = 16 / (int)sizeof(T);
    auto s16 = [&](int j) { return j >= 0 && j % VE == 0 && j >= lo && j + VE - 1 <= hi; };
    auto s8 = [&](int j) {
        return sizeof(T) == 4 && j >= 0 && j % 2 == 0 && j >= lo && j + 1 <= hi && !s16(j - j % VE);
    };
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i < lo || i > hi) continue;
        if (s16(i)) {
            if constexpr (sizeof(T) == 4) {
                const float4 q = *reinterpret_cast<const float4 *>(rowp + i);
                v[i] = q.x;
                v[i + 1] = q.y;
                v[i + 2] = q.z;
                v[i + 3] = q.w;
            } else {
                const double2 q = *reinterpret_cast<const double2 *>(rowp + i);
                v[i] = q.x;
                v[i + 1] = q.y;
            }
        } else if (s16(i - i % VE)) {
            // loaded with its 16-byte group
        } else if (s8(i)) {
            const float2 q = *reinterpret_cast<const float2 *>(reinterpret_cast<const float *>(rowp) + i);
            v[i] = (T)q.x;
            v[i + 1] = (T)q.y;
        } else if (s8(i - i % 2)) {
            // loaded with its 8-byte pair
        } else {
            v[i] = rowp[i];
        }
    }
}

template <typename T, int SHAPE, int R>
__global__ void __launch_bounds__(kThreads, 2)
    cu3d_stream(const T *__restrict__ in, T *__restrict__ out,
                const __grid_constant__ Weights<T, Taps<SHAPE, 3, R>::K> wt, int64_t Ez, int64_t Ey, int64_t Ex,
                int tiles_x, int tiles_y, int chunks_z, int nitems)
{
    constexpr int KT = Taps<SHAPE, 3, R>::K;
    constexpr bool kSmemW = sizeof(T) == 8;
    constexpr int RPT = stream_rows_per_thread<T>(), BY = 16 * RPT, BX = 64;
    constexpr int PW = stream_pitch<T, R>(), PH = BY + 2 * R, PE = stream_plane_elems<T, R>();
    constexpr int PF = stream_prefetch<T, R>();
    constexpr int NP = 2 * R + 1 + PF;
    constexpr int VE = 16 / (int)sizeof(T);  // elements per 16 bytes
    constexpr int NV = 4 + 2 * R;            // row segment of a thread
    constexpr int NL = (NV + VE - 1) / VE;   // 16-byte loads per row segment
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *wsm = reinterpret_cast<T *>(smem_raw);
    if (kSmemW) {
        for (int k = threadIdx.x; k < KT; k += blockDim.x) wsm[k] = wt.w[k];
    }
    T *ring = reinterpret_cast<T *>(smem_raw + (kSmemW ? (KT * sizeof(T) + 15) / 16 * 16 : 0));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15, x0 = 4 * tx;
    const int64_t nz = Ez - 2 * R, ny = Ey - 2 * R, nx = Ex - 2 * R;
    // rows start on 16-byte boundaries in global memory when the stored row
    // length is a 16-byte multiple and `in` is aligned (the staged window of
    // every tile starts at column 64 bx, a 16-byte multiple)
    const bool vec = (Ex * (int64_t)sizeof(T)) % 16 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % tiles_x, by = (item / tiles_x) % tiles_y, bz = item / (tiles_x * tiles_y);
        // stored coordinates of the first output of the item
        const int64_t Z0 = R + (int64_t)bz * kStreamCZ, Y0 = R + (int64_t)by * BY, X0 = R + (int64_t)bx * BX;
        const int64_t rem = nz - (Z0 - R);
        const int nzo = (int)(rem < kStreamCZ ? rem : kStreamCZ);  // output planes of this item
        const int64_t zfirst = Z0 - R;                                // first input plane
        const int nin = nzo + 2 * R;                                  // input planes of the item
        // copy input plane gz (rows Y0-R.., columns X0-R.., zero outside the
        // stored grid) into its ring slot
        auto load_plane = [&](int64_t gz) {
            T *dst = ring + (size_t)((gz - zfirst) % NP) * PE;
            const bool zok = gz >= 0 && gz < Ez;
            for (int row = warp; row < PH; row += kThreads / 32) {
                const int64_t gy = Y0 - R + row;
                const bool rok = zok && gy >= 0 && gy < Ey;
                const T *src = in + ((rok ? gz : 0) * Ey + (rok ? gy : 0)) * Ex;
                for (int c = lane * VE; c < PW; c += 32 * VE) {
                    const int64_t gx = X0 - R + c;
                    if (vec && rok && gx + VE <= Ex) {
                        cp_async_elem<16>(dst + row * PW + c, src + gx, true);
                    } else {
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            const bool ok = rok && gx + e < Ex;
                            cp_async_elem<sizeof(T)>(dst + row * PW + c + e, ok ? src + gx + e : in, ok);
                        }
                    }
                }
            }
        };
        __syncthreads();  // the previous item's reads of the ring are done
        // planes 0 .. 2R (the first output's) and the PF planes after them
        for (int k = 0; k < 2 * R + 1; ++k) load_plane(zfirst + k);
        cp_async_commit();
#pragma unroll
        for (int f = 0; f < PF; ++f) {
            if (2 * R + 1 + f < nin) load_plane(zfirst + 2 * R + 1 + f);
            cp_async_commit();
        }
        for (int zo = 0; zo < nzo; ++zo) {
            // planes zo .. zo + 2R are needed: all but the PF newest groups
            cp_async_wait_group<PF>();
            __syncthreads();
            T acc[RPT][4];
#pragma unroll
            for (int i = 0; i < RPT; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = T(0);
#pragma unroll
            for (int oz = -R; oz <= R; ++oz) {
                const T *pl = ring + (size_t)((zo + R + oz) % NP) * PE;
#pragma unroll
                for (int oy = -R; oy <= R; ++oy) {
                    bool any = false;
#pragma unroll
                    for (int ox = -R; ox <= R; ++ox) any = any || tap_index<SHAPE, 3, R>(oz, oy, ox) >= 0;
                    if (!any) continue;
#pragma unroll
                    for (int i = 0; i < RPT; ++i) {
                        const T *rowp = pl + (ty + 16 * i + R + oy) * PW + x0;
                        T v[NL * VE];
                        load_seg<T, NL * VE>(rowp, v, seg_lo<SHAPE, R>(oz, oy), seg_hi<SHAPE, R>(oz, oy));
#pragma unroll
                        for (int ox = -R; ox <= R; ++ox) {
                            const int k = tap_index<SHAPE, 3, R>(oz, oy, ox);
                            if (k >= 0) {
                                const T wk = kSmemW ? wsm[k] : wt.w[k];
#pragma unroll
                                for (int c = 0; c < 4; ++c) acc[i][c] = fma(wk, v[c + R + ox], acc[i][c]);
                            }
                        }
                    }
                }
            }
            const int64_t gz = Z0 + zo;
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int64_t gy = Y0 + ty + 16 * i;
                if (gy - R >= ny) continue;
                T *orow = out + (gz * Ey + gy) * Ex;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int64_t gx = X0 + x0 + c;
                    if (gx - R < nx) orow[gx] = acc[i][c];
                }
            }
            __syncthreads();  // plane zo is no longer read: its slot takes plane zo + 2R + 1 + PF
            if (zo + 2 * R + 1 + PF < nin) load_plane(zfirst + zo + 2 * R + 1 + PF);
            cp_async_commit();
        }
    }
    cp_async_wait_group<0>();
}


// ---------------------------------------------------------------------------
// 3-D, t = 1, FP32: z-marching with rotating partial sums.
// ---------------------------------------------------------------------------
// A work item is a 64-column x BY-row tile and a run of cz output planes.
// The CTA stages ONE input plane at a time (a ring of kRotNPL planes keeps the
// next ones in flight with cp.async) and adds it, once, into every output
// plane it touches: input plane ip contributes its 2-D slice w(oz, ., .) to
// output plane ip - R - oz for oz in [-R, R], so each thread keeps the partial
// sums of its 4 columns x RPT rows for 2R+1 output planes in registers
// (slots rotate with the plane index; the plane loop is unrolled by 2R+1, so
// every slot and weight index is a compile-time constant).  Output plane oq
// is complete after input plane oq + 2R and is stored from its slot.  Input
// planes of the first and last 2R of a run also add into slots of outputs
// outside the run; those slots are cleared, never stored.
// Staged planes hold columns X0 - 4 .. X0 + 67 (tiles start R mod 4 columns
// left of the interior, so the window and every thread's 4 output columns
// are 16-byte aligned): a thread's taps need the 16-byte chunks tx, tx+1,
// tx+2 of a row; rows that only the centre column touches (star stencils)
// need chunk tx+1 alone.  Each staged value is read from shared memory once
// per (row, thread) instead of once per output plane.
constexpr int kRotNPL = 4;   // ring planes: the one computed and three in flight
constexpr int kRotPW = 72;   // staged columns (64 + 2 x 4)

template <int SHAPE, int R>
__host__ __device__ constexpr int rot_rows_per_thread()
{
    return R <= 2 ? 2 : 1;
}

template <int SHAPE, int R>
__host__ __device__ constexpr size_t rot_smem_bytes()
{
    return (size_t)kRotNPL * (16 * rot_rows_per_thread<SHAPE, R>() + 2 * R) * kRotPW * sizeof(float);
}

// Does staged row j (0 .. RPT + 2R - 1) of a thread need more than the
// centre chunk?  (Yes if some output row i takes it as its own row, oy = 0,
// or the stencil is a box.)
template <int SHAPE, int R, int RPT>
__host__ __device__ constexpr bool rot_full_row(int j)
{
    return SHAPE == 0 || (j >= R && j < R + RPT);
}

template <int SHAPE, int R>
__global__ void __launch_bounds__(kThreads, 2)  // 2 CTAs per SM: the unrolled planes take 80-115 registers
    cu3d_rot(const float *__restrict__ in, float *__restrict__ out,
             const __grid_constant__ Weights<float, Taps<SHAPE, 3, R>::K> wt, int64_t Ez, int64_t Ey, int64_t Ex,
             int tiles_x, int tiles_y, int nitems, int cz, int xs)
{
    constexpr int RPT = rot_rows_per_thread<SHAPE, R>(), BY = 16 * RPT, BX = 64;
    constexpr int PH = BY + 2 * R, PW = kRotPW, PE = PH * PW, NS = 2 * R + 1;
    constexpr int NCH = PW / 4;  // 16-byte chunks per staged row
    static_assert(R <= 3, "the plane loop unrolls (2R+1)-fold: radii up to 3");
    extern __shared__ __align__(16) float ring[];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t nz = Ez - 2 * R, ny = Ey - 2 * R, nx = Ex - 2 * R;
    const bool vec = (Ex & 3) == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const bool vst = (Ex & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;

    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % tiles_x, by = (item / tiles_x) % tiles_y, bz = item / (tiles_x * tiles_y);
        // stored coordinates of the item's first output (column X0 may lie in the halo)
        const int64_t Z0 = R + (int64_t)bz * cz, Y0 = R + (int64_t)by * BY, X0 = R + (int64_t)bx * BX - xs;
        const int64_t rem = nz - (Z0 - R);
        const int nzo = (int)(rem < cz ? rem : cz);
        const int nin = nzo + 2 * R;
        const int64_t zfirst = Z0 - R;
        // items whose staged rows and columns lie inside the stored plane (all
        // but the edges): 32-bit in-plane offsets, no per-chunk tests
        const bool inner = vec && Y0 - R >= 0 && Y0 - R + PH <= Ey && X0 - 4 >= 0 && X0 - 4 + PW <= Ex;
        const int ex32 = (int)Ex;                        // a stored row holds < 2^31 values
        const int base_off = (int)((Y0 - R) * Ex + (X0 - 4));  // and a stored plane too
        auto load_plane = [&](int ip) {
            float *dst = ring + (size_t)(ip & (kRotNPL - 1)) * PE;
            const int64_t gz = zfirst + ip;
            const bool zok = gz >= 0 && gz < Ez;
            if (inner && zok) {
                const float *src = in + gz * Ey * Ex + base_off;
                for (int e = tid; e < PH * NCH; e += kThreads) {
                    const int row = e / NCH, ch = e - (e / NCH) * NCH;
                    cp_async_elem<16>(dst + row * PW + 4 * ch, src + row * ex32 + 4 * ch, true);
                }
                return;
            }
            for (int e = tid; e < PH * NCH; e += kThreads) {
                const int row = e / NCH, ch = e - (e / NCH) * NCH;
                const int64_t gy = Y0 - R + row, gx = X0 - 4 + 4 * ch;
                const bool rok = zok && gy >= 0 && gy < Ey;
                const float *src = in + ((rok ? gz : 0) * Ey + (rok ? gy : 0)) * Ex;
                float *d = dst + row * PW + 4 * ch;
                if (vec) {
                    // gx is a multiple of 4 and so is Ex: the chunk is wholly in or out
                    const bool ok = rok && gx >= 0 && gx < Ex;
                    cp_async_elem<16>(d, ok ? src + gx : in, ok);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const bool ok = rok && gx + c >= 0 && gx + c < Ex;
                        cp_async_elem<4>(d + c, ok ? src + gx + c : in, ok);
                    }
                }
            }
        };
        __syncthreads();  // the previous item's reads of the ring are done
#pragma unroll
        for (int k = 0; k < kRotNPL - 1; ++k) {
            if (k < nin) load_plane(k);
            cp_async_commit();
        }
        float acc[NS][RPT][4];
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int i = 0; i < RPT; ++i) acc[s][i][0] = acc[s][i][1] = acc[s][i][2] = acc[s][i][3] = 0.0f;
        const int64_t gy0 = Y0 + ty * RPT, gx0 = X0 + 4 * tx;
        // this thread's output quads: offset within a stored plane, row inside
        // the interior, and which columns are interior
        const bool qfull = gx0 >= R && gx0 + 3 - R < nx;
        unsigned cmask = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) cmask |= (gx0 + c >= R && gx0 + c - R < nx) ? (1u << c) : 0u;
        const int nrow_ok = (int)min((int64_t)RPT, ny + R - gy0);  // rows of the thread inside the interior
        const int ooff0 = (int)(gy0 * Ex + gx0);                  // offset within a stored plane
        for (int base = 0; base < nin; base += NS) {
            // the NS planes of this round; u is a compile-time constant, so every
            // accumulator slot index below is one too (no run-time selects)
            static_for<NS>([&](auto U) -> bool {
                constexpr int u = decltype(U)::value;
                const int ip = base + u;
                if (ip >= nin) return false;
                // plane ip + NPL - 1 goes into the slot plane ip - 1 used (read before the last barrier)
                if (ip + kRotNPL - 1 < nin) load_plane(ip + kRotNPL - 1);
                cp_async_commit();
                cp_async_wait_group<kRotNPL - 1>();  // plane ip has landed
                __syncthreads();
                const float *pl = ring + (size_t)(ip & (kRotNPL - 1)) * PE + (ty * RPT) * PW + 4 * tx;
#pragma unroll
                for (int j = 0; j < RPT + 2 * R; ++j) {
                    const float *rowp = pl + j * PW;
                    float v[12];
                    const float4 c1 = *reinterpret_cast<const float4 *>(rowp + 4);
                    v[4] = c1.x;
                    v[5] = c1.y;
                    v[6] = c1.z;
                    v[7] = c1.w;
                    if (rot_full_row<SHAPE, R, RPT>(j)) {
                        const float4 c0 = *reinterpret_cast<const float4 *>(rowp);
                        const float4 c2 = *reinterpret_cast<const float4 *>(rowp + 8);
                        v[0] = c0.x;
                        v[1] = c0.y;
                        v[2] = c0.z;
                        v[3] = c0.w;
                        v[8] = c2.x;
                        v[9] = c2.y;
                        v[10] = c2.z;
                        v[11] = c2.w;
                    }
#pragma unroll
                    for (int i = 0; i < RPT; ++i) {
                        const int oy = j - i - R;
                        if (oy < -R || oy > R) continue;
#pragma unroll
                        for (int oz = -R; oz <= R; ++oz) {
                            const int slot = ((u - R - oz) % NS + 2 * NS) % NS;
#pragma unroll
                            for (int ox = -R; ox <= R; ++ox) {
                                const int k = tap_index<SHAPE, 3, R>(oz, oy, ox);
                                if (k >= 0) {
#pragma unroll
                                    for (int c = 0; c < 4; ++c)
                                        acc[slot][i][c] = fmaf(wt.w[k], v[4 + c + ox], acc[slot][i][c]);
                                }
                            }
                        }
                    }
                }
                // output plane ip - 2R is complete (slot (u + 1) mod NS)
                const int oq = ip - 2 * R;
                constexpr int sd = (u + 1) % NS;
                if (oq >= 0 && oq < nzo) {
                    float *obase = out + (Z0 + oq) * Ey * Ex;
#pragma unroll
                    for (int i = 0; i < RPT; ++i) {
                        if (i >= nrow_ok) continue;
                        float *o = obase + ooff0 + i * ex32;
                        if (vst && qfull) {
                            *reinterpret_cast<float4 *>(o) =
                                make_float4(acc[sd][i][0], acc[sd][i][1], acc[sd][i][2], acc[sd][i][3]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if ((cmask >> c) & 1u) o[c] = acc[sd][i][c];
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < RPT; ++i) acc[sd][i][0] = acc[sd][i][1] = acc[sd][i][2] = acc[sd][i][3] = 0.0f;
                __syncthreads();  // the slot of plane ip is free for plane ip + NPL
                return true;
            });
        }
    }
    cp_async_wait_group<0>();
}

}  // namespace cu
}  // namespace gbs
