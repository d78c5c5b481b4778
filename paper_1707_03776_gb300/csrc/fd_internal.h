// Internal types shared by the host API (fd_api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fd.h"

namespace fdgb {

constexpr int kMaxHalfWidth = 8;  // SO <= 16

// Three-axis view of a grid: a 2D grid (n0, n1) is the single plane
// (1, n0, n1) with the plane axis not differentiated.  Axis 2 is contiguous.
struct Geom {
    int ndim;          // 2 or 3
    int64_t n[3];      // interior extents in the 3-axis view
    int64_t s0, s1;    // strides (elements) of axes 0 and 1; axis 2 stride is 1
};

// FD coefficients of one operator: coef[a][k] = w_k / h_a^2 (FP64 -> FP32
// once), axis a in the 3-axis view (coef[0] all zero for 2D grids), and the
// summed centre weight centre = sum_a w_0 / h_a^2.
struct Coef {
    float centre;
    float ax[3][kMaxHalfWidth + 1];
};

// Linear-interpolation table of a sparse object on the device.
struct SparseDev {
    int npoint;
    int ncorner;             // 4 (2D) or 8 (3D)
    const int64_t *base;     // [npoint] linear index of the lowest corner
    const float *weight;     // [npoint][8]
    int64_t corner_off[8];   // linear offset of corner k from base
};

// ---- launchers (kernel files) -------------------------------------------

cudaError_t launch_coefficients(const Geom &g, const float *m, const float *eta, double dt,
                                float *c, float *d, cudaStream_t st);
cudaError_t launch_min_reduce(const Geom &g, const float *m, unsigned int *out_bits,
                              cudaStream_t st);
cudaError_t launch_interpolate(const SparseDev &sp, const float *u, float *out_row,
                               cudaStream_t st);
// loads the interpolation kernel's module on the current device
cudaError_t prepare_interpolate();
cudaError_t launch_inject(const SparseDev &sp, const float *c, const float *row, float *u,
                          cudaStream_t st);

// plain kernels: one thread per (d1, d2) column, streaming d0
// reads u (u^n) and up (u^{n-1}), writes out (u^{n+1}); out may equal up
cudaError_t launch_acoustic_plain(int half_width, const Geom &g, const Coef &cf,
                                  const float *u, const float *up, float *out, const float *c,
                                  const float *d, cudaStream_t st);
// grad += scale * mu * (u0 - 2 u1 + u2)
cudaError_t launch_imaging(const Geom &g, float scale, const float *mu, const float *u0,
                           const float *u1, const float *u2, float *grad, cudaStream_t st);
cudaError_t launch_imaging_steps(const Geom &g, float scale, int k, const float *const *mu, const float *const *u,
                                 float *grad, cudaStream_t st);
cudaError_t launch_diffusion_plain(int half_width, const Geom &g, const Coef &cf, float adt,
                                   const float *u, float *u_out, cudaStream_t st);

// plain 2D kernels of the Linear Convection and Laplace examples
// upwind: out = u - nux (u - u[i-1,j]) - nuy (u - u[i,j-1]), zero halo
cudaError_t launch_convection_plain(const Geom &g, float nux, float nuy, const float *u, float *out,
                                    cudaStream_t st);
// Jacobi sweep with the Dirichlet rows and Neumann columns; if sum is not
// null, *sum += sum of |out| (FP64)
cudaError_t launch_jacobi_plain(const Geom &g, float wr, float wc, const float *p, float *out, double *sum,
                                cudaStream_t st);
// sum += sum of |u| over the interior (FP64)
cudaError_t launch_abs_sum(const Geom &g, const float *u, double *sum, cudaStream_t st);

// Whole runs of small 2D grids in one thread-block cluster (k_cluster.cu)
enum { kRuleDiffusion = 0, kRuleUpwind = 1, kRuleJacobi = 2 };
struct ClusterPlan {
    bool ok = false;
    int rule = 0;
    int M = 1;        // stencil half-width
    int nctas = 0;    // CTAs in the cluster
    int K = 1;        // steps between halo exchanges
    int halo = 0;     // halo rows per side
    size_t smem = 0;  // dynamic shared memory per CTA
};
// Plan a rule on a 2D grid; want_k > 0 forces the steps per exchange.
// Returns false when the grid does not fit in a cluster.
bool cluster_plan_build(int rule, int half_width, const Geom &g, int want_k, ClusterPlan *out);
// nt steps from u0 (slot t0 % 2); the last two states go to slot0/slot1 by
// time parity.  Jacobi with tol > 0 stops on the L1 criterion; res_steps /
// res_r (device, may be null) receive the steps done and the last r.
cudaError_t launch_cluster_run(const ClusterPlan &p, const Geom &g, const Coef &cf, float adt, float nux,
                               float nuy, float wr, float wc, const float *u0, float *slot0, float *slot1,
                               long long t0, long long nt, double tol, long long *res_steps, double *res_r,
                               cudaStream_t st);

}  // namespace fdgb
