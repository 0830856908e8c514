// model.cpp -- stencil patterns, the composite kernel and the paper's
// performance model, used by the dispatcher (host only).
//
// Model (arxiv 2603.00477): K and C = 2K, M = 2D, I = K/D (Sec. 3.2.1);
// CUDA cores with temporal fusion: I_CU = tK/D, P = min(P_CU, B I) (Eq. 8);
// tensor cores with kernel fusion: alpha = K^(t)/(tK) (Eq. 9), box
// K^(t) = (2rt+1)^d (Eq. 10), I_TC = t (alpha/S) K/D and
// P_TC,actual = (S/alpha) min(P_TC, B I_TC) (Eq. 11-12); speed-up, the four
// scenarios and the sweet spot (Sec. 4.1, Eqs. 13-19); sparse tensor cores
// keep I and raise the peak (Sec. 4.3, Eq. 20).  beta (products issued per
// useful product of a split-precision form) is this library's extension and
// multiplies the issued work like alpha/S.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace gbs {

int pattern_points(int shape, int d, int r)
{
    if (shape == STENCIL_BOX) {
        int k = 1;
        for (int i = 0; i < d; i++) k *= 2 * r + 1;
        return k;
    }
    return 2 * d * r + 1;
}

bool make_pattern(int shape, int d, int r, Pattern *p)
{
    if ((shape != STENCIL_BOX && shape != STENCIL_STAR) || d < 1 || d > 3 || r < 1) return false;
    p->shape = shape;
    p->d = d;
    p->r = r;
    p->offs.clear();
    const int side = 2 * r + 1;
    int total = 1;
    for (int i = 0; i < d; i++) total *= side;
    for (int idx = 0; idx < total; idx++) {
        int c[3] = {0, 0, 0};
        int rem = idx;
        int nz = 0;
        for (int i = d - 1; i >= 0; i--) {
            c[i] = rem % side - r;
            rem /= side;
        }
        for (int i = 0; i < d; i++) nz += c[i] != 0;
        if (shape == STENCIL_STAR && nz > 1) continue;
        for (int i = 0; i < d; i++) p->offs.push_back(c[i]);
    }
    p->K = (int)(p->offs.size() / d);
    return true;
}

std::vector<double> compose_dense(const Pattern &p, const std::vector<double> &w, int t)
{
    const int d = p.d, r = p.r, R = t * r, side = 2 * R + 1;
    size_t total = 1;
    for (int i = 0; i < d; i++) total *= (size_t)side;
    std::vector<double> cur(total, 0.0), nxt(total, 0.0);
    size_t centre = 0;
    for (int i = 0; i < d; i++) centre = centre * side + R;
    cur[centre] = 1.0;
    for (int s = 0; s < t; s++) {
        std::fill(nxt.begin(), nxt.end(), 0.0);
        for (size_t idx = 0; idx < total; idx++) {
            if (cur[idx] == 0.0) continue;
            int c[3] = {0, 0, 0};
            size_t rem = idx;
            for (int i = d - 1; i >= 0; i--) {
                c[i] = (int)(rem % side) - R;
                rem /= side;
            }
            for (int k = 0; k < p.K; k++) {
                size_t q = 0;
                bool in = true;
                for (int i = 0; i < d; i++) {
                    int v = c[i] + p.offs[k * d + i];
                    if (v < -R || v > R) in = false;
                    q = q * side + (size_t)(v + R);
                }
                if (in) nxt[q] += cur[idx] * w[k];
            }
        }
        cur.swap(nxt);
    }
    return cur;
}

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    double v = 1;
    for (int i = 1; i <= k; i++) v = v * (n - k + i) / i;
    return v;
}

// Box: (2rt+1)^d (Eq. 10).  Star: the t-fold sum of star offsets is
// { p : sum_i ceil(|p_i|/r) <= t }, of size sum_j C(d,j) C(t,j) (2r)^j.
int fused_points(int shape, int d, int r, int t)
{
    if (shape == STENCIL_BOX) {
        int k = 1;
        for (int i = 0; i < d; i++) k *= 2 * r * t + 1;
        return k;
    }
    double s = 0;
    for (int j = 0; j <= std::min(d, t); j++) s += binom(d, j) * binom(t, j) * std::pow(2.0 * r, j);
    return (int)std::lround(s);
}

ModelOut model_eval(int shape, int d, int r, int t, int D, double S, double beta, double P_cu,
                    double P_tc, double B)
{
    ModelOut m;
    m.K = pattern_points(shape, d, r);
    m.K_fused = fused_points(shape, d, r, t);
    m.alpha = (double)m.K_fused / ((double)t * m.K);
    const double C = 2.0 * m.K;
    m.M = 2.0 * D;
    m.C_cu = t * C;
    m.C_tc = beta * m.alpha / S * m.C_cu;
    m.I_cu = m.C_cu / m.M;
    m.I_tc = m.C_tc / m.M;
    m.ridge_cu = P_cu / B;
    m.ridge_tc = P_tc / B;
    m.P_cu_actual = std::min(P_cu, B * m.I_cu);
    m.P_tc_actual = S / (m.alpha * beta) * std::min(P_tc, B * m.I_tc);
    m.speedup = m.P_tc_actual / m.P_cu_actual;
    const bool cu_cb = m.I_cu >= m.ridge_cu;
    const bool tc_cb = m.I_tc >= m.ridge_tc;
    m.scenario = cu_cb ? (tc_cb ? 4 : 3) : (tc_cb ? 2 : 1);
    const bool cond = m.alpha * beta < S * P_tc / P_cu;  // Eq. 19
    m.sweet_spot = (m.scenario == 3) || (m.scenario == 4 && cond);
    m.gst_cu = m.P_cu_actual / C / 1e9;
    m.gst_tc = m.P_tc_actual / C / 1e9;
    return m;
}

// GB300 defaults.  FP64 and FP32 FMA rates: 152 SMs at the 2070 MHz maximum
// clock, 2 FP64 and 128 FP32 FMA lanes per SM per clock (2 FLOP each); FP64
// MMA at the same rate as the FP64 pipe; dense TF32 1.1 and BF16 2.25
// PFLOP/s; 2:4 sparse twice dense; HBM 6.8 TB/s measured copy bandwidth.
static stencil_peaks g_peaks = {
    6.8e12,                    // hbm_bytes_per_s
    152.0 * 2.07e9 * 2 * 2,    // cu_f64_flops
    152.0 * 2.07e9 * 128 * 2,  // cu_f32_flops
    152.0 * 2.07e9 * 2 * 2,    // tc_f64_flops
    1.1e15,                    // tc_tf32_flops
    2.25e15,                   // tc_bf16_flops
    2.2e15,                    // sptc_tf32_flops
    4.5e15,                    // sptc_bf16_flops
};

// The table is process-wide and may be replaced while other threads create
// plans: every access copies it under this lock.
static std::mutex g_peaks_mutex;

// The eight rates, in declaration order.
static double stencil_peaks::*const kPeakFields[8] = {
    &stencil_peaks::hbm_bytes_per_s, &stencil_peaks::cu_f64_flops,   &stencil_peaks::cu_f32_flops,
    &stencil_peaks::tc_f64_flops,    &stencil_peaks::tc_tf32_flops,  &stencil_peaks::tc_bf16_flops,
    &stencil_peaks::sptc_tf32_flops, &stencil_peaks::sptc_bf16_flops,
};

stencil_peaks peaks()
{
    std::lock_guard<std::mutex> lock(g_peaks_mutex);
    return g_peaks;
}

}  // namespace gbs

using namespace gbs;

extern "C" stencil_status stencil_model_predict(const stencil_model_in *in, stencil_model_out *out)
try {
    if (!in || !out) return fail(STENCIL_ERR_INVALID_ARG, "stencil_model_predict: null pointer");
    if ((in->shape != STENCIL_BOX && in->shape != STENCIL_STAR) || in->d < 1 || in->d > 3 || in->r < 1 ||
        in->t < 1 || in->dtype_bytes < 1 || !(in->sparsity > 0 && in->sparsity <= 1) || !(in->beta >= 1) ||
        !(in->P_cu > 0) || !(in->P_tc > 0) || !(in->B > 0))
        return fail(STENCIL_ERR_INVALID_ARG, "stencil_model_predict: argument out of range");
    ModelOut m = model_eval(in->shape, in->d, in->r, in->t, in->dtype_bytes, in->sparsity, in->beta, in->P_cu,
                            in->P_tc, in->B);
    out->K = m.K;
    out->K_fused = m.K_fused;
    out->alpha = m.alpha;
    out->C_cu = m.C_cu;
    out->C_tc = m.C_tc;
    out->M = m.M;
    out->I_cu = m.I_cu;
    out->I_tc = m.I_tc;
    out->ridge_cu = m.ridge_cu;
    out->ridge_tc = m.ridge_tc;
    out->P_cu_actual = m.P_cu_actual;
    out->P_tc_actual = m.P_tc_actual;
    out->speedup = m.speedup;
    out->scenario = m.scenario;
    out->sweet_spot = m.sweet_spot;
    out->gstencils_cu = m.gst_cu;
    out->gstencils_tc = m.gst_tc;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_model_predict");
}

extern "C" stencil_status stencil_set_peaks(const stencil_peaks *p)
try {
    if (!p) return fail(STENCIL_ERR_INVALID_ARG, "stencil_set_peaks: null pointer");
    for (auto f : kPeakFields) {
        if (!(p->*f >= 0) || std::isinf(p->*f))
            return fail(STENCIL_ERR_INVALID_ARG, "stencil_set_peaks: a rate is negative or not finite");
    }
    std::lock_guard<std::mutex> lock(g_peaks_mutex);
    for (auto f : kPeakFields)
        if (p->*f > 0) g_peaks.*f = p->*f;
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_set_peaks");
}

extern "C" stencil_status stencil_get_peaks(stencil_peaks *p)
try {
    if (!p) return fail(STENCIL_ERR_INVALID_ARG, "stencil_get_peaks: null pointer");
    *p = peaks();
    return STENCIL_OK;
} catch (...) {
    return gbs::abi_exception("stencil_get_peaks");
}
