// tc_layout.h -- geometry of the tensor-core (Toeplitz) formulation, shared by
// the dispatcher (which reports the sparsity factor S, paper Sec. 2.2.2) and
// the launchers (which issue exactly the MMAs counted here).
//
// The t-step composite kernel w^(t) of radius R = t*r is applied as a sum
// over its rows ("lines"; in 3-D over (plane,row) pairs): for line a,
//     out[y][x0 + n] += sum_k In[y + a][x0 - R + k] * B_a[k][n],
//     B_a[k][n] = w^(t)[a][k - n - R]   (zero outside |k - n - R| <= h_a),
// a GEMM whose M axis runs over output rows y, whose N axis is a window of
// n_tile output columns and whose K axis is the input window of
// n_tile + 2R columns, padded to the MMA K step.  Line a only needs the
// K blocks that touch its band |b| <= h_a; the others are skipped.
// S = useful MACs / issued MACs = sum_a (2 h_a + 1) / sum_a (issued K of a).
#pragma once

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace gbs {

struct TcLines {
    int R = 0, n_tile = 8, k_inst = 8, kext = 0, nkb = 0;
    std::vector<int> half;          // h_a per line (2R+1 lines in 2-D), -1 = empty line
    std::vector<int> kb_lo, kb_hi;  // K-block range issued per line (lo > hi: none)
    double useful = 0, issued = 0;  // per output point
    double sparsity() const { return issued > 0 ? useful / issued : 0.0; }
};

// Half-width of line a (2-D) of the composite: a box line spans R; a star
// line spans r (t - ceil(|a|/r)) (the t-fold star sum is the set of p with
// sum_i ceil(|p_i|/r) <= t).
inline int composite_half(int shape, int r, int t, int a)
{
    const int R = t * r;
    if (shape == 0) return R;
    const int ca = (std::abs(a) + r - 1) / r;
    return ca > t ? -1 : r * (t - ca);
}

inline TcLines tc_lines_2d(int shape, int r, int t, int n_tile, int k_inst)
{
    TcLines L;
    L.R = t * r;
    L.n_tile = n_tile;
    L.k_inst = k_inst;
    L.kext = (n_tile + 2 * L.R + k_inst - 1) / k_inst * k_inst;
    L.nkb = L.kext / k_inst;
    for (int a = -L.R; a <= L.R; a++) {
        const int h = composite_half(shape, r, t, a);
        L.half.push_back(h);
        if (h < 0) {
            L.kb_lo.push_back(1);
            L.kb_hi.push_back(0);
            continue;
        }
        // non-zero k: R - h <= k <= R + h + n_tile - 1
        const int lo = (L.R - h) / k_inst;
        const int hi = std::min(L.nkb - 1, (L.R + h + n_tile - 1) / k_inst);
        L.kb_lo.push_back(lo);
        L.kb_hi.push_back(hi);
        L.useful += 2 * h + 1;
        L.issued += (double)(hi - lo + 1) * k_inst;
    }
    return L;
}

// MMA N (output columns per Toeplitz block) of the warp-specialised TF32 /
// TF32x3 kernel: the widest of 32, 16, 8 whose operands fit in 227 KB of
// shared memory -- B blocks (x2 split) plus double-buffered A tiles (hi, and
// lo when split) of 128 + 2R rows (rounded up to 8) by (NACC-1)*N + kext columns.
inline int tc_ws_ntile(int shape, int r, int t, bool split)
{
    const int R = t * r;
    const int hs = (128 + 2 * R + 7) / 8 * 8;  // chunk columns 128-byte aligned (TMA destinations)
    const int cand[3][2] = {{32, 2}, {16, 2}, {8, 4}};
    for (auto &c : cand) {
        const int n = c[0], nacc = c[1];
        TcLines L = tc_lines_2d(shape, r, t, n, 8);
        const long a = (long)((n * (nacc - 1) + L.kext) / 4) * hs * 16;
        const long b = (long)(2 * R + 1) * L.nkb * (n / 8) * 256;
        const long smem = 128 + b * (split ? 2 : 1) + a * (split ? 4 : 2);
        if (smem <= 227 * 1024) return n;
    }
    return 8;
}

// Wide FP16 kernel (tc2d_wide): the Toeplitz factor of line a is the A
// operand over M = 128 output columns (stored in reverse order, so that
// A[m'][k] depends on k + m' only) and K = 16 nkb window columns,
// nkb = ceil((128 + 2R) / 16); the input tile is the B operand over N = nr
// output rows.  Line a's A operand for every K block is read from one strip
// of 2 nkb + 15 core matrices (128 bytes each), non-zero only in core
// matrices 15 .. (127 + 2R) / 8, so consecutive lines' strips are placed
// max(2 nkb, (127 + 2R) / 8 + 1) core matrices apart and overlap in zeros.
struct WideGeom {
    int nkb, strip_len, delta, hs, nbuf;
    size_t strip_bytes, in_bytes, smem;
};

inline WideGeom tc_wide_geom(int R, int nr, bool split, int nbuf = 2)
{
    WideGeom g;
    g.nkb = (128 + 2 * R + 15) / 16;
    g.strip_len = 2 * g.nkb + 15;
    g.delta = std::max(2 * g.nkb, (127 + 2 * R) / 8 + 1);
    g.hs = (nr + 2 * R) | 1;  // odd chunk-column height: conflict-free staging stores
    g.nbuf = nbuf;
    g.strip_bytes = (size_t)(2 * R * g.delta + g.strip_len) * 128;
    g.in_bytes = (size_t)(2 * g.nkb) * g.hs * 16;
    // 1 KB header, weight strips (hi, lo), nbuf input buffers (hi, lo)
    g.smem = 1024 + (g.strip_bytes + nbuf * g.in_bytes) * (split ? 2 : 1);
    return g;
}

// Tile of the wide kernel: output rows (MMA N) and input buffers -- the
// first of (256, 2), (128, 2), (128, 1) whose operands fit in 227 KB (double
// buffering overlaps the next tile's conversion with this tile's MMAs; one
// buffer keeps N = 128 for the hi + lo forms at R = 7 .. 12).  Every R <= 12
// fits; nr = 0 beyond.
struct WideTile {
    int nr = 0, nbuf = 0;
};

inline WideTile tc_wide_tile(int r, int t, bool split)
{
    WideTile w;
    if (t * r > 12) return w;
    const int cand[3][2] = {{256, 2}, {128, 2}, {128, 1}};
    for (auto &c : cand)
        if (tc_wide_geom(t * r, c[0], split, c[1]).smem <= 227 * 1024) {
            w.nr = c[0];
            w.nbuf = c[1];
            return w;
        }
    return w;
}

// Output rows per tile (MMA N) of the wide kernel, 0 if no tile fits.
inline int tc_wide_nrows(int r, int t, bool split) { return tc_wide_tile(r, t, split).nr; }

// 3-D wide FP16 kernel (tc3d_wide, one step per sweep): the Toeplitz factor
// of line (dz, dy) is the A operand as in tc2d_wide (one strip per line, two
// strip sets: the weights are rescaled per output plane), the input is
// staged one plane tile of nr + 2R rows at a time into a ring of 2R + 2
// slots.  Lines: the (dz, dy) pairs with a non-zero weight, (2r+1)^2 for a
// box and 4r + 1 for a star.
struct Wide3Geom {
    int nkb, delta, hs, slots;
    size_t strip_bytes, in_bytes, smem;
};

inline int tc_wide3_lines(int shape, int r) { return shape == 0 ? (2 * r + 1) * (2 * r + 1) : 4 * r + 1; }  // 0: box

inline Wide3Geom tc_wide3_geom(int R, int nlines, int nr)
{
    Wide3Geom g;
    g.nkb = (128 + 2 * R + 15) / 16;
    g.delta = std::max(2 * g.nkb, (127 + 2 * R) / 8 + 1);
    g.hs = (nr + 2 * R) | 1;
    g.slots = 2 * R + 2;
    g.strip_bytes = (size_t)((nlines - 1) * g.delta + 2 * g.nkb + 15) * 128;
    g.in_bytes = (size_t)(2 * g.nkb) * g.hs * 16;
    // 1 KB header, two strip sets, the ring of input slots
    g.smem = 1024 + 2 * g.strip_bytes + (size_t)g.slots * g.in_bytes;
    return g;
}

// Output rows per tile of the 3-D kernel: the first of 128, 64, 32 whose
// operands fit in 227 KB; 0 if none does or r > 3.
inline int tc_wide3_nrows(int shape, int r)
{
    if (r < 1 || r > 3) return 0;
    for (int nr : {128, 64, 32})
        if (tc_wide3_geom(r, tc_wide3_lines(shape, r), nr).smem <= 227 * 1024) return nr;
    return 0;
}

// ---------------------------------------------------------------------------
// 2:4-structured sparse form (paper Sec. 4.3), TF32 1:2 on mma.sp m16n8k16.
//
// The sparse operand must be A, so the Toeplitz block of line a is the A
// operand: A_a[m][k] = w^(t)[a][k - m] (0 <= k - m <= 2R) with M = 16 output
// columns and K = the 16 + 2R input columns of the window; B is the im2col
// of the input (K x 8 output rows).  TF32 sparsity keeps one element of every
// pair of consecutive logical K positions, so K is permuted ("strided
// swapping"): the window is cut into 16-byte chunks (4 columns) and chunk c is
// paired with a chunk at least ceil((2R+1)/4) chunks away, so no row's band
// holds both members of a pair.  Instruction s takes the chunk pairs 2s and
// 2s+1; its logical pair p is element p/2 of chunk pair 2s + (p mod 2).  A
// chunk index of -1 is a dummy (zero operand).
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
#define GBS_HD __host__ __device__ __forceinline__
#else
#define GBS_HD inline
#endif

constexpr int kSpMaxNs = 4;  // instructions per line (R <= 12)

struct SpLayout {
    int R = 0, nc = 0, ns = 0, sigma = 0, pitch_q = 0, rl = 0;
    int cf[2 * kSpMaxNs], cs[2 * kSpMaxNs];  // chunk pairs (first, second); -1 = dummy
    int bchunk[4 * kSpMaxNs];                // chunk each lane class q of instruction s loads B from
                                             // (a dummy gets a filler chunk; its A is zero)
    std::vector<int> mask;                   // per line: bit s = instruction s issued
    double useful = 0, issued = 0;           // per output point (issued: logical K)
    double sparsity() const { return issued > 0 ? useful / issued : 0.0; }
};

// Round an FP32 value to TF32 (nearest, ties away from zero), as the
// conversion instruction does for finite values.
GBS_HD float tf32_round(float x)
{
    union {
        float f;
        unsigned u;
    } v;
    v.f = x;
    v.u = (v.u + 0x1000u) & 0xFFFFE000u;
    return v.f;
}

// Value and selector (0: first, 1: second member) of compressed A element
// (row m, logical pair p) of instruction s for line a.  w: the composite
// kernel, (2R+1) x (2R+1) row-major.
GBS_HD float sp_a_value(const double *w, int R, const int *cf, const int *cs, int a, int s, int m, int p,
                        int *sel)
{
    const int cp = 2 * s + (p & 1), i = p >> 1, lines = 2 * R + 1;
    const int fc = cf[cp], sc = cs[cp];
    *sel = 0;
    if (fc >= 0) {
        const int b = 4 * fc + i - m;
        if (b >= 0 && b <= 2 * R && w[a * lines + b] != 0.0) return tf32_round((float)w[a * lines + b]);
    }
    if (sc >= 0) {
        const int b = 4 * sc + i - m;
        if (b >= 0 && b <= 2 * R && w[a * lines + b] != 0.0) {
            *sel = 1;
            return tf32_round((float)w[a * lines + b]);
        }
    }
    return 0.0f;
}

inline SpLayout sp_layout_2d(int shape, int r, int t)
{
    SpLayout L;
    const int R = t * r;
    L.R = R;
    L.nc = (16 + 2 * R + 3) / 4;
    const int dc = (2 * R + 1 + 3) / 4;  // minimum chunk distance of a pair
    std::vector<int> pf, ps, used(L.nc, 0);
    for (int c = 0; c < L.nc; c++) {
        if (used[c]) continue;
        used[c] = 1;
        int partner = -1;
        for (int c2 = c + dc; c2 < L.nc; c2++)
            if (!used[c2]) {
                partner = c2;
                used[c2] = 1;
                break;
            }
        pf.push_back(c);
        ps.push_back(partner);
    }
    L.ns = ((int)pf.size() + 1) / 2;
    for (int i = 0; i < 2 * kSpMaxNs; i++) {
        L.cf[i] = i < (int)pf.size() ? pf[i] : -1;
        L.cs[i] = i < (int)ps.size() ? ps[i] : -1;
    }
    // B chunk of lane class q (0..3) of instruction s: first / second member
    // of chunk pair 2s + q/2.  Rows 8 apart XOR their 16-byte chunk index
    // with sigma; sigma and the filler chunks of dummies are chosen so that
    // the eight 16-byte loads of a quarter warp (two rows, four chunks) hit
    // eight distinct bank groups where possible.
    int best = 1 << 30;
    for (int sg = 0; sg < 8; sg++) {
        int total = 0, pick[4 * kSpMaxNs];
        for (int s = 0; s < L.ns; s++) {
            const int fixed[4] = {L.cf[2 * s], L.cs[2 * s], L.cf[2 * s + 1], L.cs[2 * s + 1]};
            int bestc = 1 << 30, choice[4] = {0, 0, 0, 0};
            // enumerate fillers for the dummy slots (nc <= 10 choices each)
            int slots[4], nd = 0;
            for (int j = 0; j < 4; j++)
                if (fixed[j] < 0) slots[nd++] = j;
            int combos = 1;
            for (int j = 0; j < nd; j++) combos *= L.nc;
            for (int cidx = 0; cidx < combos; cidx++) {
                int c[4], v = cidx;
                for (int j = 0; j < 4; j++) c[j] = fixed[j];
                for (int j = 0; j < nd; j++) {
                    c[slots[j]] = v % L.nc;
                    v /= L.nc;
                }
                int cnt[8] = {0};
                for (int j = 0; j < 4; j++) {
                    cnt[c[j] & 7]++;
                    cnt[(c[j] & 7) ^ sg]++;
                }
                int conf = 0;
                for (int b = 0; b < 8; b++) conf += cnt[b] > 1 ? cnt[b] - 1 : 0;
                if (conf < bestc) {
                    bestc = conf;
                    for (int j = 0; j < 4; j++) choice[j] = c[j];
                }
            }
            total += bestc;
            for (int j = 0; j < 4; j++) pick[4 * s + j] = choice[j];
        }
        if (total < best) {
            best = total;
            L.sigma = sg;
            for (int i = 0; i < 4 * L.ns; i++) L.bchunk[i] = pick[i];
        }
    }
    L.rl = 48 + 4 * L.nc;                 // staged row: 3 strips of 16 + the last window
    L.pitch_q = (L.rl / 4 + 7) / 8 * 8;  // 16-byte chunks per row, multiple of 8
    for (int a = -R; a <= R; a++) {
        const int h = composite_half(shape, r, t, a);
        int m = 0;
        if (h >= 0) {
            // non-zero columns of the line over the 16 rows: [R-h, R+h+15]
            for (int s = 0; s < L.ns; s++) {
                bool hit = false;
                for (int j = 0; j < 2; j++) {
                    const int cp = 2 * s + j;
                    for (int c : {L.cf[cp], L.cs[cp]}) {
                        if (c < 0) continue;
                        if (4 * c + 3 >= R - h && 4 * c <= R + h + 15) hit = true;
                    }
                }
                if (hit) m |= 1 << s;
            }
            L.useful += 2 * h + 1;
            L.issued += 16.0 * __builtin_popcount((unsigned)m);
        }
        L.mask.push_back(m);
    }
    return L;
}

}  // namespace gbs
