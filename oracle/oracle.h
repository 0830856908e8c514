/*
 * oracle.h -- plain FP64 CPU oracle for repeated star/box stencil sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The GPU
 * product path never links, loads or calls it, and this file shares no code
 * with the product (package paper_2603_00477_gb300/).
 *
 * What it computes (paper Sec. 1, the stencil definition; Sec. 3.2.1 for K):
 *   every interior grid point takes the weighted sum of a fixed neighbour
 *   pattern; box = every offset in [-r, r]^d, star = offsets with at most one
 *   non-zero coordinate.  Grids are stored with a fixed (Dirichlet) halo of
 *   width r around the interior, row-major, last axis contiguous.  One step:
 *       v[p] = sum_{o in O} w_o * u[p + o]      for every interior p,
 *   halo cells copied unchanged.  O is ordered lexicographically, first axis
 *   outermost, each coordinate ascending from -r; weights follow that order.
 *   The sum is formed in that order in FP64 (compiled with -ffp-contract=off).
 *
 * Temporal fusion (paper Sec. 2.2.3, kernel fusion; Eq. 9-10 for the fused
 * support): t steps equal one application of the t-fold self-convolution
 * w^(t) (radius t*r) at points whose fused neighbourhood does not cross the
 * fixed halo.  oracle_compose builds w^(t) as a dense (2tr+1)^d box.
 *
 * Conventions: shape 0 = box, 1 = star.  d in {1,2,3}.  dims[] are interior
 * extents, slowest axis first; stored extents are dims[i] + 2r.  All
 * functions return 0 on success and a negative value on a bad argument.
 * nthreads <= 0 means "OpenMP default".
 */
#ifndef STENCIL_ORACLE_H
#define STENCIL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Number of offsets K of the pattern: box (2r+1)^d, star 2dr+1. */
int oracle_num_offsets(int shape, int d, int r);

/* Writes the K offsets (K*d ints, offset-major) in O order.  Returns K. */
int oracle_offsets(int shape, int d, int r, int *offs);

/* One step from u to v (both stored arrays with halo width r). */
int oracle_step(int shape, int d, int r, const double *w, const int64_t *dims,
                const double *u, double *v, int nthreads);

/* `steps` stepwise steps, in place on u (stored array with halo). */
int oracle_run(int shape, int d, int r, const double *w, const int64_t *dims,
               double *u, int64_t steps, int nthreads);

/* Dense composite kernel w^(t) of radius R = t*r: (2R+1)^d values, box order
 * (lexicographic, first axis outermost).  t = 0 gives the identity kernel. */
int oracle_compose(int shape, int d, int r, const double *w, int t, double *wt);

/* One application of a dense radius-R kernel to a stored array with halo
 * width `halo`, at interior points at least `margin` away from the interior
 * boundary (needs R <= margin + halo).  Other points of v are left as set by
 * the caller. */
int oracle_apply_dense(int d, int R, const double *wk, int halo,
                       const int64_t *dims, const double *u, double *v,
                       int margin, int nthreads);

/* `steps` stepwise steps evaluated only where needed to produce the interior
 * box [lo, hi) (interior coordinates, slowest axis first).  u_full is the
 * whole stored initial field (with halo), left unchanged.  out receives the
 * box, row-major.  Cost is that of the dependency cone of the box. */
int oracle_run_region(int shape, int d, int r, const double *w,
                      const int64_t *dims, const double *u_full, int64_t steps,
                      const int64_t *lo, const int64_t *hi, double *out,
                      int nthreads);

/* Threads an OpenMP parallel region gets with nthreads <= 0. */
int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
