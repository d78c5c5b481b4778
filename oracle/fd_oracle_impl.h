/*
 * Body of the CPU oracle, written once and included twice by fd_oracle.c:
 * once with REAL = double (suffix _f64) and once with REAL = float (suffix _f32).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this.
 *
 * Conventions (all arrays dense row-major, no halo stored):
 *   ndim = 3: fields have shape (n0, n1, n2), axis a has spacing h[a].
 *   ndim = 2: fields have shape (n0, n1); internally handled as (1, n0, n1)
 *             with only the last two axes differentiated.
 *   Values outside [0, n_a) on any axis are zero (zero Dirichlet halo).
 *   Sparse traces are time-major: trace[n * npoint + p].
 */

#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)
#define FN(name) CAT(name, SUFFIX)

/* Field value with the zero halo: u(i0, i1, i2), zero when any index is
 * outside the grid.  This is the ghost-node reading of the boundary. */
static REAL FN(val_)(const REAL *u, const int64_t *N, int64_t i0, int64_t i1, int64_t i2)
{
    if (i0 < 0 || i0 >= N[0] || i1 < 0 || i1 >= N[1] || i2 < 0 || i2 >= N[2])
        return (REAL)0;
    return u[(i0 * N[1] + i1) * N[2] + i2];
}

/* Laplacian (the paper's `u.laplace`, Seismic Inversion Example): the sum over
 * every space axis of the central second-derivative stencil of half-width M,
 *   (L u)_i = sum_a (1/h_a^2) sum_{k=-M..M} w_{|k|} u_{i + k e_a},
 * with u = 0 outside the grid. coef[a][k] holds w_k / h_a^2 in REAL. */
static void FN(laplacian_)(int ndim, const int64_t *N, int M, REAL coef[3][17],
                           const REAL *u, REAL *Lu)
{
    int first_axis = 3 - ndim;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t i0 = 0; i0 < N[0]; i0++)
        for (int64_t i1 = 0; i1 < N[1]; i1++)
            for (int64_t i2 = 0; i2 < N[2]; i2++) {
                REAL sum = 0;
                for (int a = first_axis; a < 3; a++) {
                    for (int k = -M; k <= M; k++) {
                        int kk = k < 0 ? -k : k;
                        int64_t j0 = i0 + (a == 0 ? k : 0);
                        int64_t j1 = i1 + (a == 1 ? k : 0);
                        int64_t j2 = i2 + (a == 2 ? k : 0);
                        sum += coef[a][kk] * FN(val_)(u, N, j0, j1, j2);
                    }
                }
                Lu[(i0 * N[1] + i1) * N[2] + i2] = sum;
            }
}

/* Stencil coefficients w_k / h_a^2, from the closed-form weights in FP64,
 * rounded once to REAL. */
static int FN(stencil_coef_)(int ndim, const double *spacing, int space_order, REAL coef[3][17])
{
    double w[9];
    if (or_weights_central2(space_order, w) != 0) return -1;
    int M = space_order / 2;
    memset(coef, 0, sizeof(REAL) * 3 * 17);
    for (int d = 0; d < ndim; d++) {
        int a = 3 - ndim + d;
        double h = spacing[d];
        for (int k = 0; k <= M; k++) coef[a][k] = (REAL)(w[k] / (h * h));
    }
    return 0;
}

/* Receiver interpolation (the paper's `rec.interpolate(expr=u)`):
 * out[p] = sum over the 2^ndim surrounding nodes of weight * u(node). */
static void FN(interpolate_)(int ndim, const int64_t *N, const OrTable *tab,
                             const REAL *u, REAL *out)
{
    int ncorner = 1 << ndim;
    for (int p = 0; p < tab->npoint; p++) {
        REAL s = 0;
        for (int c = 0; c < ncorner; c++) {
            const int64_t *ix = &tab->node[((int64_t)p * 8 + c) * 3];
            s += (REAL)tab->weight[(int64_t)p * 8 + c] * u[(ix[0] * N[1] + ix[1]) * N[2] + ix[2]];
        }
        out[p] = s;
    }
}

/* Source injection (the paper's `src.inject(field=u, expr=src*dt**2/m)`):
 * u(node) += weight * (dt^2 / m(node)) * value[p], with dt^2/m taken at the
 * node being written (coefficient array c = dt^2/m). */
static void FN(inject_)(int ndim, const int64_t *N, const OrTable *tab,
                        const REAL *c, const REAL *value, REAL *u)
{
    int ncorner = 1 << ndim;
    for (int p = 0; p < tab->npoint; p++) {
        for (int k = 0; k < ncorner; k++) {
            const int64_t *ix = &tab->node[((int64_t)p * 8 + k) * 3];
            int64_t at = (ix[0] * N[1] + ix[1]) * N[2] + ix[2];
            u[at] += (REAL)tab->weight[(int64_t)p * 8 + k] * c[at] * value[p];
        }
    }
}

/* Coefficient fields of the acoustic update: c = dt^2/m and d = dt*eta/m
 * (solving m u_tt + eta u_t - lap u = q for u(t+dt) with a centred second
 * and a backward first time difference). */
static void FN(coefficients_)(int64_t n, const float *m, const float *eta, double dt,
                              REAL *c, REAL *d)
{
    REAL dtr = (REAL)dt;
    for (int64_t i = 0; i < n; i++) {
        c[i] = dtr * dtr / (REAL)m[i];
        d[i] = (eta ? dtr * (REAL)eta[i] / (REAL)m[i] : (REAL)0);
    }
}

/* Forward acoustic modelling (Seismic Inversion Example, forward operator).
 * Time step n (t_n = n dt) for n = t0 .. t0+nt-1, in this order:
 *   1. rec[n] = R u^n                                  (interpolate)
 *   2. u^{n+1} = 2u^n - u^{n-1} + c L u^n - d (u^n - u^{n-1})
 *   3. u^{n+1} += c Q^T src[n]                         (inject)
 * On entry u_cur = u^{t0}, u_prev = u^{t0-1}; on exit u_cur = u^{t0+nt},
 * u_prev = u^{t0+nt-1}.  src/rec traces are [n_total][npoint]. */
int FN(or_acoustic_forward)(int ndim, const int64_t *shape, const double *spacing,
                            const double *origin, int space_order,
                            const float *m, const float *eta, double dt,
                            int64_t t0, int64_t nt, REAL *u_cur, REAL *u_prev,
                            int nsrc, const double *src_coords, const REAL *src_trace,
                            int nrec, const double *rec_coords, REAL *rec_trace)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    REAL coef[3][17];
    if (FN(stencil_coef_)(ndim, spacing, space_order, coef) != 0) return -1;
    int M = space_order / 2;
    int64_t n = N[0] * N[1] * N[2];
    REAL *c = (REAL *)malloc(sizeof(REAL) * n);
    REAL *d = (REAL *)malloc(sizeof(REAL) * n);
    REAL *Lu = (REAL *)malloc(sizeof(REAL) * n);
    REAL *unew = (REAL *)malloc(sizeof(REAL) * n);
    OrTable src = {0, NULL, NULL}, rec = {0, NULL, NULL};
    int rc = (c && d && Lu && unew) ? 0 : -2;
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nsrc, src_coords, &src);
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nrec, rec_coords, &rec);
    if (rc != 0) {
        or_table_free_(&src); or_table_free_(&rec);
        free(c); free(d); free(Lu); free(unew);
        return rc;
    }
    FN(coefficients_)(n, m, eta, dt, c, d);

    for (int64_t step = t0; step < t0 + nt; step++) {
        if (nrec > 0) FN(interpolate_)(ndim, N, &rec, u_cur, rec_trace + step * nrec);
        FN(laplacian_)(ndim, N, M, coef, u_cur, Lu);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            unew[i] = 2 * u_cur[i] - u_prev[i] + c[i] * Lu[i] - d[i] * (u_cur[i] - u_prev[i]);
        if (nsrc > 0) FN(inject_)(ndim, N, &src, c, src_trace + step * nsrc, unew);
        memcpy(u_prev, u_cur, sizeof(REAL) * n);
        memcpy(u_cur, unew, sizeof(REAL) * n);
    }
    or_table_free_(&src); or_table_free_(&rec);
    free(c); free(d); free(Lu); free(unew);
    return 0;
}

/* Adjoint acoustic modelling (Seismic Inversion Example, adjoint operator).
 * This is the exact transpose of or_acoustic_forward over steps 0..nt-1
 * started from rest.  Writing the adjoint state as mu = C lambda (C = diag c),
 * the transpose of the forward recurrence is, for n = nt-1 down to 0,
 *   1. srca[n] = Q mu^{n+1}                            (interpolate at sources)
 *   2. mu^n = 2mu^{n+1} - mu^{n+2} + c L mu^{n+1} - d (mu^{n+1} - mu^{n+2})
 *   3. mu^n += c R^T r[n]                              (inject receiver data)
 * with mu^{nt} = mu^{nt+1} = 0: the forward update run backward in time, with
 * the roles of the two point sets swapped, as the paper prescribes. */
int FN(or_acoustic_adjoint)(int ndim, const int64_t *shape, const double *spacing,
                            const double *origin, int space_order,
                            const float *m, const float *eta, double dt, int64_t nt,
                            int nrec, const double *rec_coords, const REAL *rec_trace,
                            int nsrc, const double *src_coords, REAL *srca_trace,
                            REAL *mu_out /* mu^0 on exit, may be NULL */)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    REAL coef[3][17];
    if (FN(stencil_coef_)(ndim, spacing, space_order, coef) != 0) return -1;
    int M = space_order / 2;
    int64_t n = N[0] * N[1] * N[2];
    REAL *c = (REAL *)malloc(sizeof(REAL) * n);
    REAL *d = (REAL *)malloc(sizeof(REAL) * n);
    REAL *Lmu = (REAL *)malloc(sizeof(REAL) * n);
    REAL *mu1 = (REAL *)calloc(n, sizeof(REAL)); /* mu^{n+1} */
    REAL *mu2 = (REAL *)calloc(n, sizeof(REAL)); /* mu^{n+2} */
    REAL *mu0 = (REAL *)malloc(sizeof(REAL) * n); /* mu^{n}   */
    OrTable src = {0, NULL, NULL}, rec = {0, NULL, NULL};
    int rc = (c && d && Lmu && mu1 && mu2 && mu0) ? 0 : -2;
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nsrc, src_coords, &src);
    if (rc == 0) rc = or_table_build_(ndim, shape, spacing, origin, nrec, rec_coords, &rec);
    if (rc != 0) {
        or_table_free_(&src); or_table_free_(&rec);
        free(c); free(d); free(Lmu); free(mu1); free(mu2); free(mu0);
        return rc;
    }
    FN(coefficients_)(n, m, eta, dt, c, d);

    for (int64_t step = nt - 1; step >= 0; step--) {
        if (nsrc > 0) FN(interpolate_)(ndim, N, &src, mu1, srca_trace + step * nsrc);
        FN(laplacian_)(ndim, N, M, coef, mu1, Lmu);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            mu0[i] = 2 * mu1[i] - mu2[i] + c[i] * Lmu[i] - d[i] * (mu1[i] - mu2[i]);
        if (nrec > 0) FN(inject_)(ndim, N, &rec, c, rec_trace + step * nrec, mu0);
        memcpy(mu2, mu1, sizeof(REAL) * n);
        memcpy(mu1, mu0, sizeof(REAL) * n);
    }
    if (mu_out) memcpy(mu_out, mu1, sizeof(REAL) * n);
    or_table_free_(&src); or_table_free_(&rec);
    free(c); free(d); free(Lmu); free(mu1); free(mu2); free(mu0);
    return 0;
}

/* Explicit Euler diffusion: u^{n+1} = u^n + a dt L u^n (the paper's `u.dt`
 * forward difference with `u.laplace`), zero Dirichlet halo.  Runs nt steps
 * in place on u. */
int FN(or_diffusion)(int ndim, const int64_t *shape, const double *spacing, int space_order,
                     double a, double dt, int64_t nt, REAL *u)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    REAL coef[3][17];
    if (FN(stencil_coef_)(ndim, spacing, space_order, coef) != 0) return -1;
    int M = space_order / 2;
    int64_t n = N[0] * N[1] * N[2];
    REAL *Lu = (REAL *)malloc(sizeof(REAL) * n);
    if (!Lu) return -2;
    REAL adt = (REAL)(a * dt);
    for (int64_t step = 0; step < nt; step++) {
        FN(laplacian_)(ndim, N, M, coef, u, Lu);
        for (int64_t i = 0; i < n; i++) u[i] = u[i] + adt * Lu[i];
    }
    free(Lu);
    return 0;
}

/* The Laplacian alone, for the oracle's own pins. */
int FN(or_laplacian)(int ndim, const int64_t *shape, const double *spacing, int space_order,
                     const REAL *u, REAL *Lu)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    REAL coef[3][17];
    if (FN(stencil_coef_)(ndim, spacing, space_order, coef) != 0) return -1;
    FN(laplacian_)(ndim, N, space_order / 2, coef, u, Lu);
    return 0;
}

/* Interpolation alone: out[p] = R u for the points given. */
int FN(or_interpolate)(int ndim, const int64_t *shape, const double *spacing,
                       const double *origin, int npoint, const double *coords,
                       const REAL *u, REAL *out)
{
    int64_t N[3];
    if (or_dims_(ndim, shape, N) != 0) return -1;
    OrTable tab;
    int rc = or_table_build_(ndim, shape, spacing, origin, npoint, coords, &tab);
    if (rc != 0) { or_table_free_(&tab); return rc; }
    FN(interpolate_)(ndim, N, &tab, u, out);
    or_table_free_(&tab);
    return 0;
}


/* Linear convection (Linear Convection section, Eq. 2dconvdiscr): forward
 * Euler in time and backward first differences in space,
 *   u+(i,j) = u(i,j) - c dt D_x u - c dt D_y u,
 * D_a u = (w_0 u(i-1) + w_1 u(i)) / h_a with (w_0, w_1) = or_weights(1, {-1, 0}),
 * on every node of a 2D grid (x = the first axis), zero outside (zero halo).
 * nt steps in place. */
int FN(or_convection)(const int64_t *shape, const double *spacing, double c, double dt, int64_t nt, REAL *u)
{
    const int64_t nx = shape[0], ny = shape[1];
    if (nx < 1 || ny < 1) return -1;
    double off[2] = {-1.0, 0.0}, w[2];
    if (or_weights(1, 2, off, w) != 0) return -1;
    const REAL ax = (REAL)(c * dt / spacing[0]), ay = (REAL)(c * dt / spacing[1]);
    const REAL w0 = (REAL)w[0], w1 = (REAL)w[1];
    REAL *v = (REAL *)malloc(sizeof(REAL) * nx * ny);
    if (!v) return -2;
    for (int64_t s = 0; s < nt; s++) {
        for (int64_t i = 0; i < nx; i++)
            for (int64_t j = 0; j < ny; j++) {
                const REAL uc = u[i * ny + j];
                const REAL ux = i > 0 ? u[(i - 1) * ny + j] : (REAL)0;
                const REAL uy = j > 0 ? u[i * ny + j - 1] : (REAL)0;
                v[i * ny + j] = uc - ax * (w0 * ux + w1 * uc) - ay * (w0 * uy + w1 * uc);
            }
        memcpy(u, v, sizeof(REAL) * nx * ny);
    }
    free(v);
    return 0;
}

/* Laplace equation section (Eq. 2dlaplace_discr): Jacobi sweeps of the
 * central second differences solved for the centre,
 *   p+(i,j) = (dy^2 (p(i+1,j) + p(i-1,j)) + dx^2 (p(i,j+1) + p(i,j-1))) / (2 (dx^2 + dy^2))
 * on the interior nodes (weights from or_weights_central2(2)), followed by the
 * boundary expressions in the order the paper's operator lists them: the
 * x = 0 and x = max rows keep their given values (Dirichlet: p = 0 and
 * p = bc_right), then p+(:,0) = p+(:,1) and p+(:,ny-1) = p+(:,ny-2)
 * (Neumann, including the corners).  With tol > 0 the sweeps stop once
 * r = |sum|p+| - sum|p|| / sum|p| < tol (sums in FP64; r = inf while sum|p|
 * = 0), at most max_iter sweeps; with tol <= 0 exactly max_iter sweeps.
 * *iters = sweeps done, *r_last = r of the last sweep. */
int FN(or_laplace)(const int64_t *shape, const double *spacing, double tol, int64_t max_iter, REAL *p,
                   int64_t *iters, double *r_last)
{
    const int64_t nx = shape[0], ny = shape[1];
    if (nx < 3 || ny < 3) return -1;
    double w2[2];
    if (or_weights_central2(2, w2) != 0) return -1;
    /* central second difference: (w1 p(-1) + w0 p(0) + w1 p(+1)) / h^2 = 0 solved for p(0) */
    const double hx2 = spacing[0] * spacing[0], hy2 = spacing[1] * spacing[1];
    const double den = -w2[0] * (1.0 / hx2 + 1.0 / hy2);
    const REAL wx = (REAL)(w2[1] / hx2 / den), wy = (REAL)(w2[1] / hy2 / den);
    REAL *v = (REAL *)malloc(sizeof(REAL) * nx * ny);
    if (!v) return -2;
    double s_old = 0.0;
    for (int64_t k = 0; k < nx * ny; k++) s_old += fabs((double)p[k]);
    int64_t it = 0;
    double r = INFINITY;
    while (it < max_iter) {
        for (int64_t i = 1; i < nx - 1; i++)
            for (int64_t j = 1; j < ny - 1; j++)
                v[i * ny + j] = wx * (p[(i + 1) * ny + j] + p[(i - 1) * ny + j]) +
                                wy * (p[i * ny + j + 1] + p[i * ny + j - 1]);
        for (int64_t j = 0; j < ny; j++) {
            v[j] = p[j];
            v[(nx - 1) * ny + j] = p[(nx - 1) * ny + j];
        }
        for (int64_t i = 0; i < nx; i++) {
            v[i * ny] = v[i * ny + 1];
            v[i * ny + ny - 1] = v[i * ny + ny - 2];
        }
        memcpy(p, v, sizeof(REAL) * nx * ny);
        it++;
        double s_new = 0.0;
        for (int64_t k = 0; k < nx * ny; k++) s_new += fabs((double)p[k]);
        r = s_old > 0.0 ? fabs(s_new - s_old) / s_old : INFINITY;
        s_old = s_new;
        if (tol > 0.0 && r < tol) break;
    }
    free(v);
    if (iters) *iters = it;
    if (r_last) *r_last = r;
    return 0;
}

#undef FN
#undef CAT
#undef CAT2
