/*
 * fd_oracle.c -- plain CPU oracle for the explicit finite-difference method of
 * "Optimised finite difference computation from symbolic equations"
 * (arXiv 1707.03776).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent reference that
 * the CUDA path is checked against.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product library never
 * links, imports or calls it, and the two share no code.
 *
 * It is deliberately slow and literal: triple loop nests over the grid, the
 * zero halo expressed as an index test, no blocking, no fusion.  Weights come
 * from the closed form of the central second-difference weights, the general
 * weights from the Taylor moment conditions solved directly, and the
 * interpolation table is built here from the coordinates in FP64.
 *
 * What each routine follows:
 *   or_weights_central2     closed form of the central 2nd-derivative weights
 *                           behind `dx2`/`laplace` (Laplace and Seismic
 *                           Inversion examples)
 *   or_weights              Taylor moment conditions for any derivative and
 *                           offsets (`dxl`, `dt`, `dt2` in the Linear
 *                           Convection and Seismic Inversion examples)
 *   or_acoustic_forward_*   forward operator of the Seismic Inversion Example:
 *                           m u_tt + eta u_t - lap u = q, with src.inject and
 *                           rec.interpolate
 *   or_acoustic_adjoint_*   adjoint operator of the same section (exact
 *                           discrete transpose, run backward in time)
 *   or_diffusion_*          explicit Euler u_t = a lap u (the `u.dt` forward
 *                           difference with `u.laplace`)
 *   or_step_points_f64      one forward update at listed points, from FP32
 *                           states, for sampled checks on large grids
 *   or_acoustic_gradient_f64  objective 1/2 |R u - d|^2 and its adjoint-state
 *                           gradient with respect to m (the adjoint of the
 *                           Seismic Inversion Example used for inversion)
 *   or_convection_*         Linear Convection section: Eq. 2dconvdiscr
 *                           (forward Euler, backward differences)
 *   or_laplace_*            Laplace equation section: Eq. 2dlaplace_discr
 *                           Jacobi sweeps with the Dirichlet and Neumann
 *                           boundary expressions and the L1 stopping rule
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Finite-difference weights                                                */
/* ------------------------------------------------------------------------ */

static double factorial_(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= (double)i;
    return f;
}

/* Central second-derivative weights of space order 2M (half-width M):
 *   w_k = 2 (-1)^{k+1} (M!)^2 / (k^2 (M-k)! (M+k)!),  k = 1..M
 *   w_0 = -2 sum_{k>=1} w_k
 * so that sum_k w_{|k|} f(x + k h) = h^2 f''(x) + O(h^{2M+2}).
 * Writes M+1 values.  Returns 0, or -1 for an odd or out-of-range order. */
int or_weights_central2(int space_order, double *w)
{
    if (space_order < 2 || space_order > 16 || (space_order % 2) != 0) return -1;
    int M = space_order / 2;
    double fm = factorial_(M);
    double s = 0.0;
    for (int k = 1; k <= M; k++) {
        double sign = (k % 2 == 1) ? 1.0 : -1.0;
        w[k] = 2.0 * sign * fm * fm / ((double)k * (double)k * factorial_(M - k) * factorial_(M + k));
        s += w[k];
    }
    w[0] = -2.0 * s;
    return 0;
}

/* Weights for derivative `deriv` at x = 0 from samples at offsets x_j (in grid
 * units): the w_j with sum_j w_j x_j^k / k! = [k == deriv] for k = 0..n-1,
 * i.e. the Taylor moment conditions, solved by Gaussian elimination with
 * partial pivoting.  Returns 0, -1 on bad input, -2 if the system is singular
 * (repeated offsets). */
int or_weights(int deriv, int n, const double *offsets, double *w)
{
    if (n < 1 || n > 32 || deriv < 0 || deriv >= n) return -1;
    double A[32][33];
    for (int k = 0; k < n; k++) {
        for (int j = 0; j < n; j++) A[k][j] = pow(offsets[j], k) / factorial_(k);
        A[k][n] = (k == deriv) ? 1.0 : 0.0;
    }
    for (int col = 0; col < n; col++) {
        int piv = col;
        for (int r = col + 1; r < n; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (fabs(A[piv][col]) < 1e-300) return -2;
        if (piv != col)
            for (int j = 0; j <= n; j++) { double t = A[col][j]; A[col][j] = A[piv][j]; A[piv][j] = t; }
        for (int r = 0; r < n; r++) {
            if (r == col) continue;
            double f = A[r][col] / A[col][col];
            for (int j = col; j <= n; j++) A[r][j] -= f * A[col][j];
        }
    }
    for (int j = 0; j < n; j++) w[j] = A[j][n] / A[j][j];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid dimensions and the linear-interpolation table                        */
/* ------------------------------------------------------------------------ */

/* Internal 3-axis view: 2D grids (n0, n1) become (1, n0, n1). */
static int or_dims_(int ndim, const int64_t *shape, int64_t *N)
{
    if (ndim == 3) { N[0] = shape[0]; N[1] = shape[1]; N[2] = shape[2]; }
    else if (ndim == 2) { N[0] = 1; N[1] = shape[0]; N[2] = shape[1]; }
    else return -1;
    for (int a = 0; a < 3; a++) if (N[a] < 1) return -1;
    return 0;
}

typedef struct {
    int npoint;
    int64_t *node;   /* [npoint][8][3] node indices in the 3-axis view */
    double *weight;  /* [npoint][8] */
} OrTable;

/* Linear (bilinear in 2D, trilinear in 3D) interpolation table, the meaning
 * of PointData's interpolate/inject: per axis s = (x - origin)/h in FP64,
 * i = floor(s) clamped to [0, n-2] (a point on the upper face puts weight 1 on
 * node n-1), f = s - i, and the 2^ndim corners get the products of f and
 * (1 - f).  Points outside [origin, origin + (n-1) h] are an error (-3). */
static int or_table_build_(int ndim, const int64_t *shape, const double *spacing,
                           const double *origin, int npoint, const double *coords,
                           OrTable *tab)
{
    tab->npoint = npoint;
    tab->node = NULL;
    tab->weight = NULL;
    if (npoint <= 0) return 0;
    tab->node = (int64_t *)calloc((size_t)npoint * 24, sizeof(int64_t));
    tab->weight = (double *)calloc((size_t)npoint * 8, sizeof(double));
    if (!tab->node || !tab->weight) return -2;
    for (int p = 0; p < npoint; p++) {
        int64_t base[3] = {0, 0, 0};
        double frac[3] = {0, 0, 0};
        for (int d = 0; d < ndim; d++) {
            int a = 3 - ndim + d;
            int64_t n = shape[d];
            double s = (coords[(int64_t)p * ndim + d] - origin[d]) / spacing[d];
            if (!(s >= 0.0) || s > (double)(n - 1) || n < 2) return -3;
            int64_t i = (int64_t)floor(s);
            if (i > n - 2) i = n - 2;
            base[a] = i;
            frac[a] = s - (double)i;
        }
        for (int c = 0; c < (1 << ndim); c++) {
            double w = 1.0;
            int64_t *ix = &tab->node[((int64_t)p * 8 + c) * 3];
            ix[0] = base[0]; ix[1] = base[1]; ix[2] = base[2];
            for (int d = 0; d < ndim; d++) {
                int a = 3 - ndim + d;
                int bit = (c >> d) & 1;
                ix[a] = base[a] + bit;
                w *= bit ? frac[a] : (1.0 - frac[a]);
            }
            tab->weight[(int64_t)p * 8 + c] = w;
        }
    }
    return 0;
}

static void or_table_free_(OrTable *tab)
{
    free(tab->node);
    free(tab->weight);
    tab->node = NULL;
    tab->weight = NULL;
}

/* Exported view of the table, for the oracle's own pins: node indices in the
 * caller's axis order ([npoint][2^ndim][ndim]) and weights ([npoint][2^ndim]). */
int or_table(int ndim, const int64_t *shape, const double *spacing, const double *origin,
             int npoint, const double *coords, int64_t *nodes_out, double *weights_out)
{
    OrTable tab;
    int rc = or_table_build_(ndim, shape, spacing, origin, npoint, coords, &tab);
    if (rc != 0) { or_table_free_(&tab); return rc; }
    int nc = 1 << ndim;
    for (int p = 0; p < npoint; p++)
        for (int c = 0; c < nc; c++) {
            for (int d = 0; d < ndim; d++)
                nodes_out[((int64_t)p * nc + c) * ndim + d] = tab.node[((int64_t)p * 8 + c) * 3 + 3 - ndim + d];
            weights_out[(int64_t)p * nc + c] = tab.weight[(int64_t)p * 8 + c];
        }
    or_table_free_(&tab);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Loop nests in FP64 and FP32                                               */
/* ------------------------------------------------------------------------ */

#define REAL double
#define SUFFIX _f64
#include "fd_oracle_impl.h"
#undef REAL
#undef SUFFIX

#define REAL float
#define SUFFIX _f32
#include "fd_oracle_impl.h"
#undef REAL
#undef SUFFIX

/* ------------------------------------------------------------------------ */
/* Sampled checks on large grids                                             */
/* ------------------------------------------------------------------------ */

/* One forward acoustic update (step 2 of or_acoustic_forward, without
 * injection) evaluated in FP64 at `npts` listed points, from FP32 states u^n
 * and u^{n-1} given densely in the (n0, n1, n2) / (n0, n1) layout:
 *   out[q] = 2u - u_prev + c L u - d (u - u_prev)  at linear index idx[q]. */
int or_step_points_f64(int ndim, const int64_t *shape, const double *spacing, int space_order,
                       const float *m, const float *eta, double dt,
                       const float *u_cur, const float *u_prev,
                       int64_t npts, const int64_t *idx, double *out)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    double w[9];
    if (or_weights_central2(space_order, w) != 0) return -1;
    int M = space_order / 2;
    int first_axis = 3 - ndim;
    double h2[3] = {1, 1, 1};
    for (int d = 0; d < ndim; d++) h2[3 - ndim + d] = spacing[d] * spacing[d];
    int64_t total = N[0] * N[1] * N[2];
    for (int64_t q = 0; q < npts; q++) {
        int64_t at = idx[q];
        if (at < 0 || at >= total) return -3;
        int64_t i0 = at / (N[1] * N[2]);
        int64_t i1 = (at / N[2]) % N[1];
        int64_t i2 = at % N[2];
        double lap = 0.0;
        for (int a = first_axis; a < 3; a++) {
            double s = 0.0;
            for (int k = -M; k <= M; k++) {
                int kk = k < 0 ? -k : k;
                int64_t j0 = i0 + (a == 0 ? k : 0);
                int64_t j1 = i1 + (a == 1 ? k : 0);
                int64_t j2 = i2 + (a == 2 ? k : 0);
                double v = 0.0;
                if (j0 >= 0 && j0 < N[0] && j1 >= 0 && j1 < N[1] && j2 >= 0 && j2 < N[2])
                    v = (double)u_cur[(j0 * N[1] + j1) * N[2] + j2];
                s += w[kk] * v;
            }
            lap += s / h2[a];
        }
        double c = dt * dt / (double)m[at];
        double d = eta ? dt * (double)eta[at] / (double)m[at] : 0.0;
        double u = (double)u_cur[at], up = (double)u_prev[at];
        out[q] = 2.0 * u - up + c * lap - d * (u - up);
    }
    return 0;
}

/* Interpolation in FP64 from an FP32 field (rec = R u), for sampled checks. */
int or_interpolate_from_f32(int ndim, const int64_t *shape, const double *spacing,
                            const double *origin, int npoint, const double *coords,
                            const float *u, double *out)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    OrTable tab;
    int rc = or_table_build_(ndim, shape, spacing, origin, npoint, coords, &tab);
    if (rc != 0) { or_table_free_(&tab); return rc; }
    int nc = 1 << ndim;
    for (int p = 0; p < npoint; p++) {
        double s = 0.0;
        for (int c = 0; c < nc; c++) {
            const int64_t *ix = &tab.node[((int64_t)p * 8 + c) * 3];
            s += tab.weight[(int64_t)p * 8 + c] * (double)u[(ix[0] * N[1] + ix[1]) * N[2] + ix[2]];
        }
        out[p] = s;
    }
    or_table_free_(&tab);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Adjoint-state gradient (FP64)                                             */
/* ------------------------------------------------------------------------ */

/* Objective and gradient of J(m) = 1/2 sum_n sum_r (rec[n][r] - d[n][r])^2
 * for the forward operator of or_acoustic_forward started from rest, with
 * m and eta given in FP64 and eta held fixed.
 *
 * The forward step is u^{n+1} = 2u^n - u^{n-1} + r^n / m with
 * r^n = dt^2 (L u^n + Q^T src[n]) - dt eta (u^n - u^{n-1}), so a change dm
 * adds -(dm/m) (u^{n+1} - 2u^n + u^{n-1}) to u^{n+1}.  Carrying that source
 * through the transpose of the recurrence (lambda, with mu = C lambda the
 * adjoint state or_acoustic_adjoint computes when the residual is injected at
 * the receivers) gives
 *   dJ/dm(x) = -(1/dt^2) sum_{n=1}^{nt-1} mu^n(x) (u^n - 2u^{n-1} + u^{n-2})(x).
 * This routine stores the whole forward history (small grids only), runs the
 * adjoint recurrence backward and sums that imaging condition.
 * grad may be NULL (objective only). */
int or_acoustic_gradient_f64(int ndim, const int64_t *shape, const double *spacing, const double *origin,
                             int space_order, const double *m, const double *eta, double dt, int64_t nt,
                             int nsrc, const double *src_coords, const double *src_trace,
                             int nrec, const double *rec_coords, const double *d_obs,
                             double *J_out, double *grad)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0 || nt < 1) return -1;
    double coef[3][17];
    if (stencil_coef__f64(ndim, spacing, space_order, coef) != 0) return -1;
    int M = space_order / 2;
    int64_t n = N[0] * N[1] * N[2];
    double *c = (double *)malloc(sizeof(double) * n);
    double *d = (double *)malloc(sizeof(double) * n);
    double *hist = (double *)calloc((size_t)(nt + 2) * n, sizeof(double)); /* u^{-1} .. u^{nt} */
    double *Lu = (double *)malloc(sizeof(double) * n);
    double *rec = (double *)calloc((size_t)nt * (nrec > 0 ? nrec : 1), sizeof(double));
    double *res = (double *)calloc((size_t)nt * (nrec > 0 ? nrec : 1), sizeof(double));
    double *mu0 = (double *)calloc(n, sizeof(double));
    double *mu1 = (double *)calloc(n, sizeof(double));
    double *mu2 = (double *)calloc(n, sizeof(double));
    OrTable src = {0, NULL, NULL}, rct = {0, NULL, NULL};
    int rc = (c && d && hist && Lu && rec && res && mu0 && mu1 && mu2) ? 0 : -2;
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nsrc, src_coords, &src);
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nrec, rec_coords, &rct);
    if (rc != 0) goto done;
    for (int64_t i = 0; i < n; i++) {
        c[i] = dt * dt / m[i];
        d[i] = eta ? dt * eta[i] / m[i] : 0.0;
    }
#define U(k) (hist + (size_t)((k) + 1) * n)
    /* forward, keeping every state; u^{-1} = u^0 = 0 */
    for (int64_t s = 0; s < nt; s++) {
        double *u = U(s), *up = U(s - 1), *un = U(s + 1);
        if (nrec > 0) interpolate__f64(ndim, N, &rct, u, rec + s * nrec);
        laplacian__f64(ndim, N, M, coef, u, Lu);
        for (int64_t i = 0; i < n; i++) un[i] = 2 * u[i] - up[i] + c[i] * Lu[i] - d[i] * (u[i] - up[i]);
        if (nsrc > 0) inject__f64(ndim, N, &src, c, src_trace + s * nsrc, un);
    }
    {
        double J = 0.0;
        for (int64_t k = 0; k < nt * nrec; k++) {
            res[k] = rec[k] - d_obs[k];
            J += 0.5 * res[k] * res[k];
        }
        *J_out = J;
    }
    if (grad) {
        for (int64_t i = 0; i < n; i++) grad[i] = 0.0;
        /* adjoint: mu^n = 2mu^{n+1} - mu^{n+2} + c L mu^{n+1} - d (mu^{n+1} - mu^{n+2}) + c R^T res[n] */
        for (int64_t s = nt - 1; s >= 0; s--) {
            laplacian__f64(ndim, N, M, coef, mu1, Lu);
            for (int64_t i = 0; i < n; i++)
                mu0[i] = 2 * mu1[i] - mu2[i] + c[i] * Lu[i] - d[i] * (mu1[i] - mu2[i]);
            if (nrec > 0) inject__f64(ndim, N, &rct, c, res + s * nrec, mu0);
            if (s >= 1) {
                const double *a = U(s), *b = U(s - 1), *e = U(s - 2);
                for (int64_t i = 0; i < n; i++) grad[i] -= mu0[i] * (a[i] - 2 * b[i] + e[i]) / (dt * dt);
            }
            double *t = mu2;
            mu2 = mu1;
            mu1 = mu0;
            mu0 = t;
        }
    }
#undef U
done:
    or_table_free_(&src);
    or_table_free_(&rct);
    free(c); free(d); free(hist); free(Lu); free(rec); free(res); free(mu0); free(mu1); free(mu2);
    return rc;
}
