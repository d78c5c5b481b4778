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
cudaError_t launch_diffusion_plain(int half_width, const Geom &g, const Coef &cf, float adt,
                                   const float *u, float *u_out, cudaStream_t st);

// whole-run diffusion in one thread-block cluster (2D grids that fit in the
// cluster's shared memory)
bool diffusion_cluster_fits(int half_width, const Geom &g, int *nclusters, size_t *smem);
cudaError_t launch_diffusion_cluster(int half_width, const Geom &g, const Coef &cf, float adt,
                                     const float *u0, float *out_last, float *out_prev, int nt,
                                     int nclusters, size_t smem, cudaStream_t st);

}  // namespace fdgb
