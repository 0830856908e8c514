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
// lo when split) of 128 + 2R rows (odd) by (NACC-1)*N + kext columns.
inline int tc_ws_ntile(int shape, int r, int t, bool split)
{
    const int R = t * r;
    const int hs = (128 + 2 * R) | 1;
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

}  // namespace gbs
