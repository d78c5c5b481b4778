/*
 * fd.h -- C ABI of the GB300-native explicit finite-difference library
 * (libfdgb.so), after "Optimised finite difference computation from symbolic
 * equations" (arXiv 1707.03776).
 *
 * The paper states the problem as: symbolic data objects that own their data
 * (TimeData, DenseData, PointData; Design and API section), an Operator built
 * from update equations and grid spacings (`Operator(..., subs={h: dx,
 * s: dt})`), applied for a number of time steps (`op(time=N)`, Linear
 * Convection section), whose data can be rebound by name (Laplace equation
 * section), and sparse points that inject into and interpolate from the grid
 * (Seismic Inversion Example).  The calls below are that statement, in C:
 *
 *   fd_weights*          FD coefficients (the `dx2`/`laplace`/`dxl`/`dt`
 *                        shorthands), FP64, host only
 *   fd_grid_*            the discretised domain: shape, spacing, origin
 *   fd_field_*           TimeData (2 time slots) / DenseData (1 slot) over
 *                        caller-owned device memory
 *   fd_sparse_*          PointData: off-grid coordinates + a device trace
 *   fd_operator_*        the Operator: build, rebind, apply for nt steps
 *
 * Conventions shared by every call:
 *   - Every call returns an fd_status; FD_OK is 0.  On failure a thread-local
 *     message is available from fd_last_error().  No C++ exception crosses
 *     this boundary.
 *   - Device memory belongs to the caller (e.g. PyTorch).  The library never
 *     frees caller memory.  Handles belong to the caller and are released with
 *     the matching *_destroy.  The library owns only its scratch: the
 *     coefficient fields c = dt^2/m and d = dt*eta/m of an acoustic operator,
 *     the interpolation tables of a sparse object and one status word per
 *     operator, allocated with cudaMallocAsync on the stream given and freed on
 *     destroy.
 *   - Work is enqueued asynchronously on the caller's CUDA stream.  Errors
 *     raised by kernels surface as FD_ERR_CUDA or FD_ERR_TIMEOUT at the next
 *     fd_operator_sync.
 *   - Floating-point data on the device is FP32.  Coordinates, spacings,
 *     weights and dt cross the boundary as FP64 host values.
 *
 * Axis convention: a grid has ndim = 2 or 3 axes (d0, d1[, d2]); the last
 * axis is contiguous in memory.  The seismic workloads map (x, y, z) to
 * (d0, d1, d2), with depth z contiguous.
 */
#ifndef FD_H
#define FD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum {
    FD_OK = 0,
    FD_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad name */
    FD_ERR_UNSUPPORTED = 2,   /* valid request this library does not implement */
    FD_ERR_LAYOUT = 3,        /* strides or alignment differ from fd_field_layout */
    FD_ERR_OUT_OF_DOMAIN = 4, /* a sparse point lies outside the grid */
    FD_ERR_UNSTABLE = 5,      /* dt above the stability limit of the scheme */
    FD_ERR_CUDA = 6,          /* a CUDA runtime or driver call failed */
    FD_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up */
    FD_ERR_NOMEM = 8          /* device or host allocation failed */
} fd_status;

/* Static English name of a status code. */
const char *fd_status_string(fd_status status);
/* Message of the last failing call on this thread ("" if none).  The pointer
 * stays valid until the next failing call on the same thread. */
const char *fd_last_error(void);
/* Library version, major*10000 + minor*100 + patch. */
int fd_version(void);

/* ------------------------------------------------------------------------
 * FD weights (host, FP64)
 * ------------------------------------------------------------------------ */

/* Weights of the derivative of order `deriv` at x = 0 from samples at the `n`
 * offsets (in grid units, distinct): sum_j w_j f(x_j) = f^(deriv)(0) h^deriv
 * + O(h^n).  These are the coefficients behind the paper's derivative
 * shorthands (`u.dxl` = offsets {-1, 0}, `u.dt` = {0, 1}, `u.dt2` =
 * {-1, 0, 1}; Linear Convection and Seismic Inversion Example sections).
 * Computed with Fornberg's recurrence (Math. Comp. 51, 1988).
 * weights_out: n doubles.  Errors: FD_ERR_INVALID_ARG for n < 1, n > 64,
 * deriv < 0 or deriv >= n, null pointers, repeated offsets. */
fd_status fd_weights(int deriv, int n, const double *offsets, double *weights_out);

/* Central second-derivative weights of even space order SO = 2M in [2, 16]:
 * w_out[k] for k = 0..M, the stencil being sum_{k=-M..M} w_{|k|} f(x + k h)
 * = h^2 f''(x) + O(h^{SO+2}) -- the `dx2` shorthand and, summed over axes,
 * `u.laplace` (Laplace equation and Seismic Inversion Example sections).
 * Errors: FD_ERR_UNSUPPORTED for odd or out-of-range orders. */
fd_status fd_weights_central2(int space_order, double *w_out);

/* ------------------------------------------------------------------------
 * Grid
 * ------------------------------------------------------------------------ */

typedef struct fd_grid fd_grid;

/* A regular grid of ndim = 2 or 3 axes with shape[a] >= 2 interior nodes,
 * spacing[a] > 0 and node 0 at origin[a] (origin may be NULL: all zero).
 * Node i of axis a sits at origin[a] + i * spacing[a].  The grid is
 * surrounded by an implicit zero halo (zero Dirichlet ghost nodes) as wide as
 * any stencil needs; nothing of the halo is stored.
 * Errors: FD_ERR_INVALID_ARG. */
fd_status fd_grid_create(int ndim, const int64_t *shape, const double *spacing,
                         const double *origin, fd_grid **out);
void fd_grid_destroy(fd_grid *grid);

/* ------------------------------------------------------------------------
 * Fields (TimeData / DenseData)
 * ------------------------------------------------------------------------ */

typedef struct fd_field fd_field;

/* Memory layout a field of this grid must have, so that the caller (e.g.
 * torch) can allocate it.  One time slot is a row-major FP32 array of
 * padded_shape (ndim entries); the last axis is padded to a multiple of 8
 * elements (32 bytes) so every row starts 32-byte aligned; pad elements are
 * never read or written.  strides[a] (in elements) and interior_offset
 * (always 0: no halo is stored) describe it.  The layout does not depend on
 * the space order; `space_order` is checked (even, 2..16) and otherwise
 * unused.  Base pointers must be 32-byte aligned. */
fd_status fd_field_layout(const fd_grid *grid, int space_order, int64_t *padded_shape,
                          int64_t *strides, int64_t *interior_offset);

/* Wrap caller-owned device memory as a field of `levels` time slots: 2 for a
 * time-dependent field (TimeData with time_order 2 or a ping-pong pair), 1 for
 * a static one (DenseData: m, eta).  dev_ptrs: `levels` device pointers, each
 * one slot in the layout of fd_field_layout (strides must be equal to it:
 * FD_ERR_LAYOUT otherwise; pass NULL to assert the layout).  Contents are not
 * touched.  The grid must outlive the field.
 * Errors: FD_ERR_INVALID_ARG, FD_ERR_LAYOUT (strides or 32-byte alignment). */
fd_status fd_field_wrap(const fd_grid *grid, int levels, void *const *dev_ptrs,
                        const int64_t *strides, fd_field **out);
void fd_field_destroy(fd_field *field);

/* ------------------------------------------------------------------------
 * Sparse points (PointData)
 * ------------------------------------------------------------------------ */

typedef struct fd_sparse fd_sparse;

/* `npoint` off-grid points with host FP64 coordinates [npoint][ndim] in the
 * grid's physical units, and a caller-owned FP32 device trace holding row n
 * (time t_n = n dt) at dev_trace + n * trace_stride, n = 0..nt-1, columns
 * 0..npoint-1 (trace_stride >= npoint).  This is the paper's PointData with
 * `data` time-major (the transpose of its (npoint, ntime) view).
 * The linear-interpolation table (bilinear in 2D, trilinear in 3D) is built
 * here in FP64 and stored on the device rounded to FP32: per axis
 * s = (x - origin)/h, i = floor(s) clamped to [0, n-2], f = s - i, the 2^ndim
 * surrounding nodes weighted by products of f and 1 - f.  The table is
 * uploaded on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 * npoint may be 0.
 * Errors: FD_ERR_INVALID_ARG (also for npoint > 0 on a grid with an axis of
 * fewer than 2 nodes, which has no interpolation cell), FD_ERR_OUT_OF_DOMAIN
 * (a point outside [origin, origin + (n-1) h] on some axis), FD_ERR_NOMEM,
 * FD_ERR_CUDA. */
fd_status fd_sparse_create(const fd_grid *grid, int npoint, const double *coords,
                           void *dev_trace, int64_t nt, int64_t trace_stride,
                           void *cuda_stream, fd_sparse **out);
/* Point the sparse object at another trace buffer of the same geometry. */
fd_status fd_sparse_set_trace(fd_sparse *sparse, void *dev_trace, int64_t nt,
                              int64_t trace_stride);
void fd_sparse_destroy(fd_sparse *sparse);

/* ------------------------------------------------------------------------
 * Operator
 * ------------------------------------------------------------------------ */

typedef struct fd_operator fd_operator;

enum {
    /* u^{n+1} = u^n + a dt L u^n: explicit Euler for u_t = a lap u (the
     * paper's `u.dt` with `u.laplace`).  u: 2 slots, ping-pong: step n reads
     * slot n%2 and writes slot (n+1)%2.  Needs `a`; m, eta, src, rec unused. */
    FD_DIFFUSION_EULER = 1,
    /* m u_tt + eta u_t - lap u = q (Seismic Inversion Example, forward
     * operator), centred second and backward first difference in time:
     *   rec[n]  = R u^n                       (rec.interpolate(expr=u))
     *   u^{n+1} = 2u^n - u^{n-1} + c L u^n - d (u^n - u^{n-1})
     *   u^{n+1} += c Q^T src[n]               (src.inject(u, src*dt^2/m))
     * with c = dt^2/m and d = dt*eta/m evaluated at each node.  u: 2 slots,
     * slot n%2 holds u^n; step n overwrites slot (n+1)%2 (u^{n-1}) with
     * u^{n+1}.  Needs m; eta, src, rec optional. */
    FD_ACOUSTIC_LEAPFROG = 2,
    /* u_t + c u_x + c u_y = 0 (Linear Convection section, Eq. 2dconvdiscr):
     *   u^{n+1} = u^n - (c dt/dx)(u^n - u^n[i-1,j]) - (c dt/dy)(u^n - u^n[i,j-1])
     * forward Euler with backward (upwind) differences, on every node of a 2D
     * grid (x = the first axis), zero halo.  space_order must be 1; `a` is the
     * velocity c > 0.  u: 2 slots, ping-pong as diffusion.  Stable (and
     * monotone) for c dt (1/dx + 1/dy) <= 1, which apply checks. */
    FD_CONVECTION_UPWIND = 3,
    /* p_xx + p_yy = 0 (Laplace equation section, Eq. 2dlaplace_discr): one
     * Jacobi sweep per step n,
     *   p^{n+1}[i,j] = (dy^2 (p[i+1,j] + p[i-1,j]) + dx^2 (p[i,j+1] + p[i,j-1]))
     *                  / (2 (dx^2 + dy^2))
     * on the interior nodes of a 2D grid, followed by the boundary expressions
     * in the paper's order: the first and last rows (x = 0 and x = max) keep
     * their values (Dirichlet: the caller stores p = 0 and p = bc_right
     * there), then the first and last columns copy the next column inwards
     * (Neumann dp/dy = 0, corners included).  space_order must be 2; dt and
     * `a` are unused.  u: 2 slots, ping-pong.  See fd_operator_converge for
     * the paper's convergence loop. */
    FD_LAPLACE_JACOBI = 4
};

enum {
    /* Run the time index backward: step n (n = t0+nt-1 down to t0) reads the
     * state of time n+1 from slot (n+1)%2 and time n+2 from slot n%2 and
     * writes time n into slot n%2, interpolating into rec[n] from the state
     * of time n+1 and injecting src[n] into the new state.  With the roles
     * of the point sets swapped (src = receiver data, rec = adjoint source)
     * this is the exact transpose of the forward run -- the paper's adjoint
     * operator with `time_axis=Backward`. */
    FD_FLAG_REVERSE = 1u << 0,
    /* Skip the stability check of fd_operator_apply. */
    FD_FLAG_NO_CFL_CHECK = 1u << 1,
    /* Use the plain one-thread-per-column kernels instead of the tiled TMA
     * kernels (same results within FP32 rounding; for comparison). */
    FD_FLAG_PLAIN_KERNELS = 1u << 2
};

typedef struct {
    int kind;              /* FD_DIFFUSION_EULER, FD_ACOUSTIC_LEAPFROG, FD_CONVECTION_UPWIND, FD_LAPLACE_JACOBI */
    int space_order;       /* even, 2..16 (convection: 1, Laplace: 2) */
    fd_field *u;           /* 2-slot time field */
    fd_field *m;           /* 1-slot square slowness (acoustic) */
    fd_field *eta;         /* 1-slot damping (acoustic, may be NULL) */
    double a;              /* diffusivity (diffusion), velocity c (convection) */
    fd_sparse *src;        /* injected points (acoustic, may be NULL) */
    fd_sparse *rec;        /* interpolated points (acoustic, may be NULL) */
    void *cuda_stream;     /* cudaStream_t all work is enqueued on */
    unsigned flags;        /* FD_FLAG_* */
} fd_op_desc;

/* Build an operator.  All fields and sparse objects must belong to grids of
 * the same shape.  For an acoustic operator this allocates the coefficient
 * fields c and d (2 FP32 slots) and reduces min(m) on the device for the
 * stability check (one stream synchronisation).
 * Errors: FD_ERR_INVALID_ARG, FD_ERR_UNSUPPORTED (kind/order/ndim),
 * FD_ERR_NOMEM, FD_ERR_CUDA. */
fd_status fd_operator_create(const fd_op_desc *desc, fd_operator **out);

/* Rebind one input by name, as the paper's `op(u=u, ...)` keyword arguments:
 * "u", "m", "eta" (obj is an fd_field*), "src", "rec" (fd_sparse*), "stream"
 * (a cudaStream_t), "a" (a const double*).  Geometry must match. */
fd_status fd_operator_bind(fd_operator *op, const char *name, void *obj);

/* Run nt >= 0 time steps n = t0 .. t0+nt-1 (the paper's `op(time=nt)`), or
 * n = t0+nt-1 down to t0 with FD_FLAG_REVERSE, with time step dt > 0.  Trace
 * rows t0..t0+nt-1 of src/rec must exist.  Enqueues the work on the
 * operator's stream and returns without waiting.  The coefficient fields are
 * recomputed when dt or m/eta changed since the last apply.
 * Errors (checked on the host before any launch): FD_ERR_INVALID_ARG,
 * FD_ERR_UNSTABLE (acoustic: dt above 2 / sqrt(max_theta lambda(theta) /
 * min m), the undamped leapfrog limit; diffusion: a dt above the explicit
 * Euler limit 2 / (a max lambda)), FD_ERR_CUDA. */
fd_status fd_operator_apply(fd_operator *op, int64_t t0, int64_t nt, double dt);

/* The Laplace example's convergence loop (FD_LAPLACE_JACOBI only): Jacobi
 * sweeps from slot t0%2 until r = |S^{n+1} - S^n| / S^n < tol, with S the sum
 * of |p| over the grid in FP64 (r is infinite while S^n = 0), or max_iter
 * sweeps.  The result is in slot (t0 + *iters) % 2.  Small grids run the
 * whole loop in one cluster launch that decides on the device; larger ones
 * read S back after every sweep.  Waits for the result.  *iters and *r_last
 * (may be NULL) receive the sweeps done and the last r.
 * Errors: FD_ERR_INVALID_ARG (tol <= 0, max_iter < 0), FD_ERR_UNSUPPORTED
 * (other kinds), FD_ERR_CUDA. */
fd_status fd_operator_converge(fd_operator *op, int64_t t0, int64_t max_iter, double tol, int64_t *iters,
                               double *r_last);

/* Temporal blocking: the loop blocking of the Devito Loop Engine (Section
 * "Automated code generation", DLE), which raises data locality to make full
 * use of the memory bandwidth, carried over to the time loop: more time steps
 * per pass over memory.
 * 2D diffusion, convection and Laplace operators: steps between halo
 * exchanges of the whole-run cluster kernel of small grids; k > 0 forces it,
 * 0 restores the planner's choice.
 * 3D acoustic operator: time steps per sweep of the grid, 1 or 2 (0: the
 * planner's choice, currently 1).  With 2, fd_operator_apply runs pairs of
 * steps in one cooperative launch (one CTA per tile column, all resident) and
 * an odd last step alone; it needs SO 4..8 and every source fused into the
 * tiled kernel.
 * Results do not depend on k (bitwise).
 * Errors: FD_ERR_UNSUPPORTED when the operator has no such path or the
 * blocking does not fit (the previous value is kept). */
fd_status fd_operator_set_time_block(fd_operator *op, int k);
/* The blocking in use: steps per exchange (2D) or per sweep (3D acoustic)
 * and the CTAs of that path (both 0 when a 2D operator runs per-step
 * kernels). */
fd_status fd_operator_get_time_block(const fd_operator *op, int *k, int *ctas);

/* Test hook of the failure path: with plane >= 0, the first tile of the tiled
 * kernel (and of the two-step kernel) never receives the copy of u^n plane
 * `plane` (its barrier is armed, the copy not issued), so that CTA's bounded
 * wait gives up after ~2 s (in the two-step kernel the other columns then
 * stop waiting on its progress as soon as they see the status),
 * records FD_ERR_TIMEOUT, drains its copies and returns; later launches do
 * nothing until fd_operator_sync reports and clears the status.  -1 turns it
 * off.  Errors: FD_ERR_UNSUPPORTED when the operator has no tiled kernel. */
fd_status fd_operator_debug_stall(fd_operator *op, int plane);

/* Wait for the operator's stream and report any deferred device error:
 * FD_ERR_CUDA for a failed launch or kernel, FD_ERR_TIMEOUT when a kernel's
 * bounded wait gave up (the status word is then cleared). */
fd_status fd_operator_sync(fd_operator *op);
void fd_operator_destroy(fd_operator *op);

/* Number of kernel launches the library has enqueued on this operator since
 * it was created (for launch accounting). */
int64_t fd_operator_launch_count(const fd_operator *op);

/* One time step between caller buffers, for schemes that keep more than two
 * states (the checkpoint recomputation of the adjoint-state gradient): the
 * update of fd_operator_apply's step n (including the operator's receiver
 * interpolation into rec[n] and source injection from src[n]) reading
 * u_cur (u^n; with FD_FLAG_REVERSE the state of time n+1) and u_prev (u^{n-1};
 * reverse: time n+2) and writing u_next (u^{n+1}; reverse: time n).  All three
 * are device FP32 slots in the layout of fd_field_layout, 32-byte aligned;
 * u_next may equal u_prev (in place) but not u_cur.  Acoustic operators only.
 * Errors: as fd_operator_apply, plus FD_ERR_LAYOUT for misaligned buffers. */
fd_status fd_operator_step(fd_operator *op, int64_t n, double dt, const void *u_cur,
                           const void *u_prev, void *u_next);

/* Imaging condition of the adjoint-state gradient with respect to m:
 * grad += scale * mu * (u0 - 2 u1 + u2) at every interior node, with mu the
 * adjoint state of time n and u0, u1, u2 the forward states of times n, n-1,
 * n-2 (device FP32 slots of `grid`'s layout, 16-byte aligned).  For
 * J(m) = 1/2 |R u - d|^2, whose adjoint is the reverse run with the residual
 * injected at the receivers, dJ/dm = -(1/dt^2) sum_n mu^n (u^n - 2u^{n-1} +
 * u^{n-2}), so scale = -1/dt^2 (an extension of the paper's adjoint operator
 * to the gradient it is built for).  Enqueued on cuda_stream.
 * Errors: FD_ERR_INVALID_ARG, FD_ERR_LAYOUT, FD_ERR_CUDA. */
fd_status fd_imaging_accumulate(const fd_grid *grid, double scale, const void *mu, const void *u0,
                                const void *u1, const void *u2, void *grad, void *cuda_stream);
/* The imaging condition above for k consecutive adjoint steps (1 <= k <= 4)
 * in one pass: for j = 0 .. k-1 in turn,
 *   grad += scale * mu[j] * (u[j] - 2 u[j+1] + u[j+2]),
 * with mu[j] the adjoint state of time n - j (k pointers) and u[i] the
 * forward state of time n - i (k + 2 pointers; host arrays of device
 * pointers).  Each forward state and grad are read once for the k steps:
 * 4 (2k + 4) bytes per node instead of 24 k.  The result equals
 * fd_imaging_accumulate for steps n, n-1, ..., n-k+1 in turn, bit for bit.
 * Same layout as fd_imaging_accumulate; grad must not alias an input.
 * Enqueued on cuda_stream.  Errors: FD_ERR_INVALID_ARG, FD_ERR_LAYOUT,
 * FD_ERR_CUDA. */
fd_status fd_imaging_accumulate_steps(const fd_grid *grid, double scale, int k, const void *const *mu,
                                      const void *const *u, void *grad, void *cuda_stream);

/* Step n of the operator (as fd_operator_apply(op, n, 1, dt)) with the
 * imaging condition above accumulated from the field the step writes:
 * grad += scale * w * (u0 - 2 u1 + u2), w the new state (with
 * FD_FLAG_REVERSE the adjoint state of time n, sources included).  This is
 * the adjoint sweep and the imaging of the gradient in one pass over the
 * grid (the paper's adjoint operator of the Seismic Inversion Example,
 * extended to the gradient it serves): the tiled kernel accumulates the
 * imaging as it writes w when it also injects the step's sources itself,
 * else the imaging kernel runs after the step (the same arithmetic, bit for
 * bit).  u0, u1, u2, grad: device FP32 slots in the layout of
 * fd_field_layout, 32-byte aligned, none a slot of the operator's field.
 * Errors: as fd_operator_apply, plus FD_ERR_LAYOUT for misaligned buffers
 * and FD_ERR_UNSUPPORTED for non-acoustic operators. */
fd_status fd_operator_apply_imaging(fd_operator *op, int64_t n, double dt, double scale, const void *u0,
                                    const void *u1, const void *u2, void *grad);

/* Tiling of the operator's tiled grid-update kernel (3D acoustic): tiles of
 * at most `rows` rows of d1 by 64 columns of d2, swept along d0, with
 * `stages` planes prefetched (2..4).  0 keeps the planner's choice for that
 * parameter.  The planner also splits d0 into chunks swept by separate CTAs
 * when the tile columns alone do not fill the GPU.   Used by the autotuner, which times candidates and keeps the
 * fastest (the GPU analogue of the paper's block-size auto-tuning, Automated
 * code generation section).  Errors: FD_ERR_UNSUPPORTED when the tiling does
 * not fit in shared memory or the operator has no tiled kernel (the previous
 * tiling is kept), FD_ERR_INVALID_ARG. */
fd_status fd_operator_set_tiling(fd_operator *op, int rows, int stages);
/* The tiling in use: rows per tile, prefetch depth, CTAs per launch (tile
 * columns x d0 chunks; all 0 when the operator runs the plain kernels). */
fd_status fd_operator_get_tiling(const fd_operator *op, int *rows, int *stages, int *ctas);
/* *fused = 1 when the tiled sweep injects the operator's sources itself (each
 * CTA stages its corners in shared memory), so that fd_operator_apply_imaging
 * also fuses the imaging condition into the sweep; 0 when injection runs as
 * its own kernel (no sources, plain kernels, or corners that would cost the
 * tiling its CTAs per SM).  Errors: FD_ERR_INVALID_ARG (null pointer). */
fd_status fd_operator_sources_fused(const fd_operator *op, int *fused);

/* Autotuner: time candidate tilings (tile heights 8..30 rows by prefetch
 * depths 2..4) over `nsteps` steps n = t0..t0+nsteps-1 with CUDA events on the
 * operator's stream and keep the fastest; writes the choice and its time per
 * step (ms) when the pointers are given.  The runs advance the operator's
 * fields and traces: tune before setting the initial state.  Synchronises the
 * stream.  Errors: FD_ERR_UNSUPPORTED (no tiled kernel), as
 * fd_operator_apply otherwise. */
fd_status fd_operator_autotune(fd_operator *op, int64_t t0, int64_t nsteps, double dt, int *best_rows,
                               int *best_stages, double *best_ms_per_step);

/* Stencil-kernel timing.  fd_operator_profile(op, n) brackets each of the
 * next n launches of the operator's grid-update kernel (the kernel that does
 * the FD update of every grid point) with CUDA events on the operator's
 * stream; n = 0 stops and discards.  fd_operator_profile_read waits for the
 * stream and returns the summed device time (ms) of the bracketed launches
 * and their number.  Errors: FD_ERR_INVALID_ARG, FD_ERR_NOMEM, FD_ERR_CUDA. */
fd_status fd_operator_profile(fd_operator *op, int64_t max_launches);
fd_status fd_operator_profile_read(fd_operator *op, double *total_ms, int64_t *launches);

/* ------------------------------------------------------------------------
 * Batches of shots
 * ------------------------------------------------------------------------ */

typedef struct fd_batch fd_batch;

/* Many forward acoustic operators (one per shot, each on its own grid, e.g. a
 * subgrid window of a larger model: the paper's forward operator applied to a
 * survey of shots) advanced together, one kernel launch per time step for all
 * of them.  All operators must be 3D, tiled (not FD_FLAG_PLAIN_KERNELS), not
 * FD_FLAG_REVERSE, of one space order and grid spacing, on one stream.  The
 * operators keep their fields, coefficients and traces; the batch sets every
 * operator's tiling to tiles of at most `rows` rows (0: 16) and sweeps with
 * `stages` planes prefetched (0: 3).  Rebinding an operator's inputs after
 * this call requires a new batch.  Errors: FD_ERR_INVALID_ARG,
 * FD_ERR_UNSUPPORTED, FD_ERR_NOMEM, FD_ERR_CUDA. */
fd_status fd_batch_create(fd_operator *const *ops, int nops, int rows, int stages, fd_batch **out);
/* Steps n = t0..t0+nt-1 of every operator (receivers, update, sources as in
 * fd_operator_apply), enqueued on the operators' stream. */
fd_status fd_batch_apply(fd_batch *batch, int64_t t0, int64_t nt, double dt);
/* Autotuner of the batch (the GPU analogue of the paper's block-size
 * auto-tuning, Automated code generation section): for tile heights of
 * 10..30 rows by prefetch depths 2..4, rebuilds the batch, runs steps
 * t0..t0+nsteps-1 of every shot timed with CUDA events on the operators'
 * stream (after up to 3 warm-up steps), and keeps the fastest; writes the
 * choice and its time per step (ms) when the pointers are given.  The runs
 * advance the shots' fields and traces: tune before setting the initial
 * state.  Drops a captured graph; synchronises the stream.  The tiling does
 * not change any result bit.  Errors: FD_ERR_UNSUPPORTED (no tiling fits),
 * FD_ERR_TIMEOUT, as fd_batch_apply. */
fd_status fd_batch_autotune(fd_batch *batch, int64_t t0, int64_t nsteps, double dt, int *best_rows,
                            int *best_stages, double *best_ms_per_step);
/* Capture steps t0..t0+nt-1 once as a CUDA graph (on a private stream; the
 * coefficients are prepared first, outside the graph), for fd_batch_replay. */
fd_status fd_batch_capture(fd_batch *batch, int64_t t0, int64_t nt, double dt);
/* Launch the captured graph on the operators' stream. */
fd_status fd_batch_replay(fd_batch *batch);
/* Wait for the stream and report deferred device errors (as fd_operator_sync). */
fd_status fd_batch_sync(fd_batch *batch);
/* Tile height, prefetch depth, CTAs per launch, launches so far. */
fd_status fd_batch_info(const fd_batch *batch, int *rows, int *stages, int *ctas, int64_t *launches);
void fd_batch_destroy(fd_batch *batch);

/* ------------------------------------------------------------------------
 * Learned closure: the 3x3x3 CNN that corrects a coarse-grid update
 * ------------------------------------------------------------------------ */

/* These calls have no counterpart in the paper: they implement a small 3D CNN
 * whose output is added to each update of a coarse-grid acoustic operator (a
 * learned closure of its discretisation error), trained on wavefields of the
 * fine-grid operator.  Activations are device BF16, channels-last with 16
 * channels per point (32 bytes), dense over a 3D shape (n0, n1, n2) with no
 * padding; smaller channel counts are zero-padded.  A layer is
 *   y[p][o] = b[o] + sum_{taps t} sum_c w[t][c][o] x[p + offset_t][c]
 * (3x3x3 cross-correlation, zero outside the grid; tap t = (a+1)*9 + (b+1)*3
 * + (c+1) for offsets a, b, c in {-1, 0, 1}), BF16 operands on the tensor
 * cores with FP32 accumulation.  All calls enqueue on cuda_stream. */

/* Pack FP32 device weights w[27][cin][cout] (cin, cout <= 16) into the
 * tensor-core operand layout frag (27 * ceil(n/8) * 256 bytes, n = cout, or
 * cin when flip = 1).  flip = 1 packs the input-gradient convolution: taps
 * mirrored and channel axes exchanged, so that fd_cnn_conv3d with it maps
 * dL/dy (cout channels) to dL/dx (cin channels). */
fd_status fd_cnn_pack_weights(const float *w, int cin, int cout, int flip, void *frag, void *cuda_stream);
/* One layer: y = relu?(conv(x, frag) + bias) [* (mask > 0)]; bias (FP32,
 * cout) may be NULL; mask (BF16 activations) may be NULL.  y_fp32 = 1 writes
 * a single linear channel as FP32 [n0*n1*n2] (cout must be 1), else BF16
 * activations.  shape: 3 int64.  x must be 16-byte, frag 8-byte, y and mask
 * 4-byte aligned (FD_ERR_LAYOUT). */
fd_status fd_cnn_conv3d(const int64_t *shape, const void *x, const void *frag, const float *bias, int cout,
                        int relu, const void *mask, void *y, int y_fp32, void *cuda_stream);
/* The same convolution on the 5th-generation tensor cores (tcgen05.mma with
 * tensor-memory accumulators, TMA-loaded planes): results equal
 * fd_cnn_conv3d's to FP32 rounding (the taps are summed in another order);
 * weights packed by fd_cnn_pack_weights_tc into 27 * 512 bytes (per (d0 tap,
 * d2 tap): [2 channel halves][48 = 3 d1 taps x 16 out][8 in] BF16).  x, y and mask must be 16-byte
 * aligned (FD_ERR_LAYOUT).  status: a device int the kernel sets to
 * FD_ERR_TIMEOUT if one of its bounded waits gave up (caller clears it).
 * Each MMA takes the three d1 taps of one (d0, d2) tap side by side in N
 * (N = 48), so a 16 -> 16 layer runs about twice as fast as fd_cnn_conv3d;
 * the closure network uses this path by default. */
fd_status fd_cnn_pack_weights_tc(const float *w, int cin, int cout, int flip, void *frag, void *cuda_stream);
fd_status fd_cnn_conv3d_tc(const int64_t *shape, const void *x, const void *frag, const float *bias, int cout,
                           int relu, const void *mask, void *y, int y_fp32, int *status, void *cuda_stream);
/* Weight and bias gradients of a layer, accumulated (+=) into FP32
 * gw[27][cin][cout] and gb[cout]: gw[t][c][o] += sum_p x[p + offset_t][c]
 * gy[p][o]. */
fd_status fd_cnn_conv3d_wgrad(const int64_t *shape, const void *x, const void *gy, int cin, int cout, float *gw,
                              float *gb, void *cuda_stream);
/* Closure inputs from a grid's fields (device FP32 slots of `grid`'s
 * fd_field_layout): with du = u - u_prev and q = 1/(m vref^2), channels 0..5
 * of x = (u, du, q u, q du, q^2 u, q^2 du) / scale, channels 6..15 = 0 (every
 * channel linear in the wavefield, so that a network without biases is
 * positively homogeneous in it).  x: BF16 activations of grid's shape.
 * noise > 0 (training): u and u_prev first get noise * xi added, xi =
 * sqrt(3) (2 r - 1) with r the top 24 bits of SplitMix64 (Steele, Lea and
 * Flood 2014) of key `seed` and counter 2p (u) or 2p + 1 (u_prev), p the
 * point's dense index (i0 n1 + i1) n2 + i2, divided by 2^24. */
fd_status fd_cnn_features(const fd_grid *grid, const float *u, const float *u_prev, const float *m, double scale,
                          double vref, double noise, uint64_t seed, void *x, void *cuda_stream);
/* The same with nsub (0..5) per-node model descriptors s_k, FP32 slots of
 * the grid's layout stored one after another from `sub` (k slots of n0
 * planes each): channels 6 + 2k and 7 + 2k are (s_k u, s_k du) / scale, still
 * linear in the wavefield.  The closure uses them for what the coarse grid's
 * sampled m does not show: the model inside a coarse cell, and the damping. */
fd_status fd_cnn_features_sub(const fd_grid *grid, const float *u, const float *u_prev, const float *m,
                              const float *sub, int nsub, double scale, double vref, double noise, uint64_t seed,
                              void *x, void *cuda_stream);
/* Injection of a fine-grid field into a coarse grid whose nodes are every
 * factor-th fine node: coarse[i, j, k] = fine[f i, f j, f k]; the fine shape
 * must be factor * (n - 1) + 1 per axis (FD_ERR_INVALID_ARG otherwise).  Both
 * are device FP32 slots of their grid's layout.  sumsq (device FP32, may be
 * NULL): += the sum of the squared coarse values. */
fd_status fd_cnn_restrict(const fd_grid *fine_grid, const float *fine, const fd_grid *coarse_grid, float *coarse,
                          int factor, float *sumsq, void *cuda_stream);
/* u += scale * corr at every interior node (corr: FP32 [n0*n1*n2]). */
fd_status fd_cnn_add_correction(const fd_grid *grid, float *u, const float *corr, double scale, void *cuda_stream);
/* Mean-squared error of pred against r = (target - base)/scale (target, base:
 * grid slots; base may be NULL for 0): *loss += mean (pred - r)^2 (FP32,
 * device), and its gradient 2 (pred - r) / count into gy (BF16 activations,
 * channel 0, the other channels zero). */
fd_status fd_cnn_mse_grad(const fd_grid *grid, const float *pred, const float *target, const float *base,
                          double scale, void *gy, float *loss, void *cuda_stream);
/* One Adam step (Kingma and Ba 2015) on n FP32 parameters with moments m1, m2
 * (step >= 1 counts from 1). */
fd_status fd_cnn_adam(float *params, const float *grads, float *m1, float *m2, int64_t n, double lr, double beta1,
                      double beta2, double eps, int64_t step, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Interpolation without allocation (the paper has no counterpart)
 * ------------------------------------------------------------------------ */

/* Largest point count fd_interpolate_noalloc accepts. */
#define FD_NOALLOC_MAX_POINTS 65536

/* Record a field at off-grid points without allocating any memory: for
 * callers that cannot call cudaMalloc when they record -- device memory fully
 * reserved up front by another allocator's pool, a fixed memory budget set at
 * start-up, or a loop that must not risk the device-wide synchronisation an
 * allocation or free can cause.  out[p] = sum of the 2^ndim linear weights of
 * point p times the field at the surrounding nodes, the same table and kernel
 * as the `rec` interpolation of fd_operator_apply.
 *   grid       grid the field belongs to
 *   coords     host FP64 [npoint][ndim], physical units, inside the grid
 *   dev_field  device FP32, one slot in the layout of fd_field_layout
 *   dev_out    device FP32 [npoint]
 *   cuda_stream  cudaStream_t the copy and the kernel are enqueued on
 * The interpolation table lives in one static device array of
 * FD_NOALLOC_MAX_POINTS entries (40 bytes each, 2.6 MB) that every GPU using
 * this call holds until the process exits; the call writes the entries it
 * uses (nothing in it needs to start at zero).  All calls on a device share
 * that array and it keeps the last call's table: calls whose work overlaps on
 * the GPU (e.g. on two streams) race.
 * Set-up: CUDA loads the library's modules lazily, so the FIRST call on a
 * device, with that device current, loads the module holding the array --
 * which allocates the array on that device and may synchronise it -- looks
 * up its device address and loads the interpolation kernel.  A call with
 * npoint = 0 does only this set-up (grid and pointers may then be NULL):
 * make it at start-up, while device memory can still be had, and before any
 * stream capture.  After it, calls on that device call no allocating routine.
 * The table reaches the device by cudaMemcpyAsync from a static pageable host
 * buffer: the call waits on the host for the stream's earlier work, and
 * concurrent callers are serialised by a lock.
 * Errors: FD_ERR_INVALID_ARG (npoint > FD_NOALLOC_MAX_POINTS or < 0, null
 * pointers), FD_ERR_OUT_OF_DOMAIN, FD_ERR_CUDA. */
fd_status fd_interpolate_noalloc(const fd_grid *grid, int npoint, const double *coords,
                                 const void *dev_field, void *dev_out, void *cuda_stream);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* FD_H */
