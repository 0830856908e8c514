/*
 * oracle.c -- plain FP64 CPU oracle for repeated star/box stencil sweeps.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h): loaded by tests/, by
 * __graft_entry__.smoke() and by the CPU legs of bench.py, never by the GPU
 * product path, with which it shares no code.
 *
 * Written to be checked by eye against the stencil definition of the paper
 * (Sec. 1: every point becomes a weighted sum of a fixed neighbour pattern;
 * box and star shapes, radius r, dimensionality d) and against the kernel
 * fusion of Sec. 2.2.3 (t steps = one sweep of the enlarged kernel of
 * radius t*r).  Every grid is handled as 3-D: a d-dimensional grid gets
 * leading axes of extent 1 without halo.  Sums run in the fixed offset order
 * in FP64; the build uses -ffp-contract=off so no FMA contraction changes the
 * rounding.  OpenMP splits the outer loops only, so results do not depend on
 * the thread count.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n[3]; /* interior extents */
    int64_t h[3]; /* halo width per axis (0 on padding axes) */
    int64_t e[3]; /* stored extents n + 2h */
} grid3;

static int make_grid(int d, int halo, const int64_t *dims, grid3 *g)
{
    if (d < 1 || d > 3 || halo < 0 || dims == NULL)
        return -1;
    int pad = 3 - d;
    for (int i = 0; i < 3; i++) {
        if (i < pad) {
            g->n[i] = 1;
            g->h[i] = 0;
        } else {
            g->n[i] = dims[i - pad];
            g->h[i] = halo;
            if (g->n[i] < 1)
                return -1;
        }
        g->e[i] = g->n[i] + 2 * g->h[i];
    }
    return 0;
}

static int64_t grid_total(const grid3 *g) { return g->e[0] * g->e[1] * g->e[2]; }

static int threads_of(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return threads_of(0); }

/* Enumerate [-r, r]^d with the last axis varying fastest (lexicographic,
 * first axis outermost); keep all of them for a box, and those with at most
 * one non-zero coordinate for a star. */
int oracle_offsets(int shape, int d, int r, int *offs)
{
    if ((shape != 0 && shape != 1) || d < 1 || d > 3 || r < 0)
        return -1;
    int side = 2 * r + 1;
    int total = 1;
    for (int i = 0; i < d; i++)
        total *= side;
    int K = 0;
    for (int idx = 0; idx < total; idx++) {
        int c[3] = {0, 0, 0};
        int rem = idx;
        for (int i = d - 1; i >= 0; i--) {
            c[i] = rem % side - r;
            rem /= side;
        }
        int nonzero = 0;
        for (int i = 0; i < d; i++)
            nonzero += (c[i] != 0);
        if (shape == 1 && nonzero > 1)
            continue;
        if (offs != NULL)
            for (int i = 0; i < d; i++)
                offs[K * d + i] = c[i];
        K++;
    }
    return K;
}

int oracle_num_offsets(int shape, int d, int r) { return oracle_offsets(shape, d, r, NULL); }

/* Linear offsets (in elements of the stored array) of the K pattern offsets. */
static int64_t *linear_offsets(int shape, int d, int r, const grid3 *g, int *K_out)
{
    int K = oracle_offsets(shape, d, r, NULL);
    if (K <= 0)
        return NULL;
    int *offs = (int *)malloc(sizeof(int) * (size_t)K * (size_t)d);
    int64_t *lin = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
    if (!offs || !lin) {
        free(offs);
        free(lin);
        return NULL;
    }
    oracle_offsets(shape, d, r, offs);
    int pad = 3 - d;
    for (int k = 0; k < K; k++) {
        int64_t o3[3] = {0, 0, 0};
        for (int i = 0; i < d; i++)
            o3[pad + i] = offs[k * d + i];
        lin[k] = (o3[0] * g->e[1] + o3[1]) * g->e[2] + o3[2];
    }
    free(offs);
    *K_out = K;
    return lin;
}

/* v[p] = sum_k w[k] * u[p + off_k] at every interior p; other cells of v
 * untouched. */
static void sweep_interior(const grid3 *g, int K, const int64_t *lin, const double *w,
                           const double *u, double *v, int nt)
{
    const int64_t e1 = g->e[1], e2 = g->e[2];
    const int64_t a0 = g->h[0], b0 = g->e[0] - g->h[0];
    const int64_t a1 = g->h[1], b1 = g->e[1] - g->h[1];
    const int64_t a2 = g->h[2], b2 = g->e[2] - g->h[2];
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
    for (int64_t i0 = a0; i0 < b0; i0++) {
        for (int64_t i1 = a1; i1 < b1; i1++) {
            for (int64_t i2 = a2; i2 < b2; i2++) {
                int64_t p = (i0 * e1 + i1) * e2 + i2;
                double acc = 0.0;
                for (int k = 0; k < K; k++)
                    acc += w[k] * u[p + lin[k]];
                v[p] = acc;
            }
        }
    }
}

int oracle_step(int shape, int d, int r, const double *w, const int64_t *dims,
                const double *u, double *v, int nthreads)
{
    grid3 g;
    if (make_grid(d, r, dims, &g) != 0 || !w || !u || !v)
        return -1;
    int K = 0;
    int64_t *lin = linear_offsets(shape, d, r, &g, &K);
    if (!lin)
        return -1;
    memcpy(v, u, sizeof(double) * (size_t)grid_total(&g)); /* halo unchanged */
    sweep_interior(&g, K, lin, w, u, v, threads_of(nthreads));
    free(lin);
    return 0;
}

int oracle_run(int shape, int d, int r, const double *w, const int64_t *dims,
               double *u, int64_t steps, int nthreads)
{
    grid3 g;
    if (make_grid(d, r, dims, &g) != 0 || !w || !u || steps < 0)
        return -1;
    if (steps == 0)
        return 0;
    int K = 0;
    int64_t *lin = linear_offsets(shape, d, r, &g, &K);
    if (!lin)
        return -1;
    size_t bytes = sizeof(double) * (size_t)grid_total(&g);
    double *tmp = (double *)malloc(bytes);
    if (!tmp) {
        free(lin);
        return -2;
    }
    memcpy(tmp, u, bytes); /* both buffers carry the same fixed halo */
    int nt = threads_of(nthreads);
    double *src = u, *dst = tmp;
    for (int64_t s = 0; s < steps; s++) {
        sweep_interior(&g, K, lin, w, src, dst, nt);
        double *x = src;
        src = dst;
        dst = x;
    }
    if (src != u)
        memcpy(u, src, bytes);
    free(tmp);
    free(lin);
    return 0;
}

/* w^(t): start from the identity (radius 0) and convolve with w t times.
 * One convolution scatters cur[c] * w_o into nxt[c + o], which is the
 * composition of two sweeps: applying w after cur reads u at p + c + o. */
int oracle_compose(int shape, int d, int r, const double *w, int t, double *wt)
{
    if (d < 1 || d > 3 || r < 0 || t < 0 || !w || !wt)
        return -1;
    int K = oracle_offsets(shape, d, r, NULL);
    if (K <= 0)
        return -1;
    int *offs = (int *)malloc(sizeof(int) * (size_t)K * (size_t)d);
    if (!offs)
        return -2;
    oracle_offsets(shape, d, r, offs);

    int R = t * r;
    int side = 2 * R + 1;
    size_t total = 1;
    for (int i = 0; i < d; i++)
        total *= (size_t)side;
    /* cur and nxt both live in the final radius-R box; cur starts as delta. */
    double *cur = (double *)calloc(total, sizeof(double));
    double *nxt = (double *)calloc(total, sizeof(double));
    if (!cur || !nxt) {
        free(offs);
        free(cur);
        free(nxt);
        return -2;
    }
    size_t centre = 0;
    for (int i = 0; i < d; i++)
        centre = centre * (size_t)side + (size_t)R;
    cur[centre] = 1.0;
    int cr = 0; /* current radius */
    for (int step = 0; step < t; step++) {
        memset(nxt, 0, total * sizeof(double));
        for (size_t idx = 0; idx < total; idx++) {
            int c[3] = {0, 0, 0};
            size_t rem = idx;
            int inside = 1;
            for (int i = d - 1; i >= 0; i--) {
                c[i] = (int)(rem % (size_t)side) - R;
                rem /= (size_t)side;
                if (c[i] < -cr || c[i] > cr)
                    inside = 0;
            }
            if (!inside || cur[idx] == 0.0)
                continue;
            for (int k = 0; k < K; k++) {
                size_t q = 0;
                for (int i = 0; i < d; i++)
                    q = q * (size_t)side + (size_t)(c[i] + offs[k * d + i] + R);
                nxt[q] += cur[idx] * w[k];
            }
        }
        double *x = cur;
        cur = nxt;
        nxt = x;
        cr += r;
    }
    memcpy(wt, cur, total * sizeof(double));
    free(offs);
    free(cur);
    free(nxt);
    return 0;
}

int oracle_apply_dense(int d, int R, const double *wk, int halo, const int64_t *dims,
                       const double *u, double *v, int margin, int nthreads)
{
    grid3 g;
    if (make_grid(d, halo, dims, &g) != 0 || R < 0 || margin < 0 || !wk || !u || !v)
        return -1;
    if (R > margin + halo)
        return -1;
    int side = 2 * R + 1;
    int total = 1;
    for (int i = 0; i < d; i++)
        total *= side;
    int64_t *lin = (int64_t *)malloc(sizeof(int64_t) * (size_t)total);
    if (!lin)
        return -2;
    int pad = 3 - d;
    for (int idx = 0; idx < total; idx++) {
        int64_t o3[3] = {0, 0, 0};
        int rem = idx;
        for (int i = d - 1; i >= 0; i--) {
            o3[pad + i] = rem % side - R;
            rem /= side;
        }
        lin[idx] = (o3[0] * g.e[1] + o3[1]) * g.e[2] + o3[2];
    }
    int64_t lo[3], hi[3];
    for (int i = 0; i < 3; i++) {
        int64_t m = (i < pad) ? 0 : margin;
        lo[i] = g.h[i] + m;
        hi[i] = g.e[i] - g.h[i] - m;
    }
    const int64_t e1 = g.e[1], e2 = g.e[2];
    int nt = threads_of(nthreads);
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
    for (int64_t i0 = lo[0]; i0 < hi[0]; i0++) {
        for (int64_t i1 = lo[1]; i1 < hi[1]; i1++) {
            for (int64_t i2 = lo[2]; i2 < hi[2]; i2++) {
                int64_t p = (i0 * e1 + i1) * e2 + i2;
                double acc = 0.0;
                for (int k = 0; k < total; k++)
                    acc += wk[k] * u[p + lin[k]];
                v[p] = acc;
            }
        }
    }
    free(lin);
    return 0;
}

int oracle_run_region(int shape, int d, int r, const double *w, const int64_t *dims,
                      const double *u_full, int64_t steps, const int64_t *lo,
                      const int64_t *hi, double *out, int nthreads)
{
    grid3 g;
    if (make_grid(d, r, dims, &g) != 0 || !w || !u_full || !lo || !hi || !out || steps < 0)
        return -1;
    int pad = 3 - d;
    int64_t blo[3], bhi[3]; /* requested box, interior coordinates */
    for (int i = 0; i < 3; i++) {
        blo[i] = (i < pad) ? 0 : lo[i - pad];
        bhi[i] = (i < pad) ? 1 : hi[i - pad];
        if (blo[i] < 0 || bhi[i] > g.n[i] || blo[i] >= bhi[i])
            return -1;
    }
    /* Window of the stored array that the dependency cone touches. */
    int64_t wlo[3], whi[3], we[3];
    for (int i = 0; i < 3; i++) {
        int64_t reach = (i < pad) ? 0 : steps * (int64_t)r;
        wlo[i] = blo[i] + g.h[i] - reach;
        whi[i] = bhi[i] + g.h[i] + reach;
        if (wlo[i] < 0)
            wlo[i] = 0;
        if (whi[i] > g.e[i])
            whi[i] = g.e[i];
        we[i] = whi[i] - wlo[i];
    }
    size_t wtotal = (size_t)(we[0] * we[1] * we[2]);
    double *A = (double *)malloc(sizeof(double) * wtotal);
    double *B = (double *)malloc(sizeof(double) * wtotal);
    int K = 0;
    int64_t *lin = NULL;
    {
        grid3 wg = g; /* linear offsets inside the window */
        wg.e[0] = we[0];
        wg.e[1] = we[1];
        wg.e[2] = we[2];
        lin = linear_offsets(shape, d, r, &wg, &K);
    }
    if (!A || !B || !lin) {
        free(A);
        free(B);
        free(lin);
        return -2;
    }
    for (int64_t i0 = 0; i0 < we[0]; i0++)
        for (int64_t i1 = 0; i1 < we[1]; i1++) {
            const double *src = u_full + ((wlo[0] + i0) * g.e[1] + (wlo[1] + i1)) * g.e[2] + wlo[2];
            memcpy(A + (i0 * we[1] + i1) * we[2], src, sizeof(double) * (size_t)we[2]);
        }
    memcpy(B, A, sizeof(double) * wtotal);
    int nt = threads_of(nthreads);
    for (int64_t s = 1; s <= steps; s++) {
        /* Points still needed after this step: the box grown by
         * (steps - s) * r, clipped to the interior (stored coordinates). */
        int64_t clo[3], chi[3];
        for (int i = 0; i < 3; i++) {
            int64_t m = (i < pad) ? 0 : (steps - s) * (int64_t)r;
            clo[i] = blo[i] + g.h[i] - m;
            chi[i] = bhi[i] + g.h[i] + m;
            if (clo[i] < g.h[i])
                clo[i] = g.h[i];
            if (chi[i] > g.e[i] - g.h[i])
                chi[i] = g.e[i] - g.h[i];
        }
#pragma omp parallel for collapse(2) schedule(static) num_threads(nt)
        for (int64_t i0 = clo[0]; i0 < chi[0]; i0++) {
            for (int64_t i1 = clo[1]; i1 < chi[1]; i1++) {
                for (int64_t i2 = clo[2]; i2 < chi[2]; i2++) {
                    int64_t p = ((i0 - wlo[0]) * we[1] + (i1 - wlo[1])) * we[2] + (i2 - wlo[2]);
                    double acc = 0.0;
                    for (int k = 0; k < K; k++)
                        acc += w[k] * A[p + lin[k]];
                    B[p] = acc;
                }
            }
        }
        double *x = A;
        A = B;
        B = x;
    }
    size_t o = 0;
    for (int64_t i0 = blo[0]; i0 < bhi[0]; i0++)
        for (int64_t i1 = blo[1]; i1 < bhi[1]; i1++)
            for (int64_t i2 = blo[2]; i2 < bhi[2]; i2++) {
                int64_t p = ((i0 + g.h[0] - wlo[0]) * we[1] + (i1 + g.h[1] - wlo[1])) * we[2] +
                            (i2 + g.h[2] - wlo[2]);
                out[o++] = A[p];
            }
    free(A);
    free(B);
    free(lin);
    return 0;
}
