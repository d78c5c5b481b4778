// Plain CUDA kernels: coefficient preparation, sparse interpolation and
// injection, and the one-thread-per-column stencil updates.
//
// The stencil kernels here are the straightforward form of the update: each
// thread owns one (d1, d2) column and walks d0, reading every neighbour from
// global memory (L1/L2 catch the reuse).  The zero halo is an index test.
#include "fd_internal.h"

namespace fdgb {

namespace {

constexpr int kThreads = 256;

// c = dt^2/m and d = dt*eta/m at every interior node (Seismic Inversion
// Example: the coefficients of u(t+dt) after solving the discretised
// m u_tt + eta u_t - lap u = q).  eta may be null (d = 0).
__global__ void coefficients_kernel(Geom g, const float *__restrict__ m,
                                    const float *__restrict__ eta, float dt2, float dt,
                                    float *__restrict__ c, float *__restrict__ d)
{
    const int64_t rows = g.n[0] * g.n[1];
    const int64_t total = rows * g.n[2];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = q / g.n[2];
        int64_t i2 = q - row * g.n[2];
        int64_t i0 = row / g.n[1];
        int64_t i1 = row - i0 * g.n[1];
        int64_t at = i0 * g.s0 + i1 * g.s1 + i2;
        float mv = m[at];
        c[at] = dt2 / mv;
        d[at] = eta ? dt * eta[at] / mv : 0.0f;
    }
}

// min over the interior of a positive field, as the order-preserving bit
// pattern of a non-negative float.
__global__ void min_reduce_kernel(Geom g, const float *__restrict__ m, unsigned int *out)
{
    const int64_t total = g.n[0] * g.n[1] * g.n[2];
    float v = 3.0e38f;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = q / g.n[2];
        int64_t i2 = q - row * g.n[2];
        int64_t i0 = row / g.n[1];
        int64_t i1 = row - i0 * g.n[1];
        float x = m[i0 * g.s0 + i1 * g.s1 + i2];
        // a non-positive or NaN entry poisons the minimum to 0
        v = (x > 0.0f) ? fminf(v, x) : 0.0f;
    }
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, __float_as_uint(v));
}

// rec[p] = sum_k w_pk u(base_p + off_k)  (rec.interpolate(expr=u))
__global__ void interpolate_kernel(SparseDev sp, const float *__restrict__ u,
                                   float *__restrict__ out)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sp.npoint) return;
    const int64_t b = sp.base[p];
    const float *w = sp.weight + (int64_t)p * 8;
    float s = 0.0f;
    for (int k = 0; k < sp.ncorner; k++) s = fmaf(w[k], u[b + sp.corner_off[k]], s);
    out[p] = s;
}

// u(base_p + off_k) += w_pk * c(node) * src[p]  (src.inject(u, src*dt^2/m));
// atomics because several points may share a node.
__global__ void inject_kernel(SparseDev sp, const float *__restrict__ c,
                              const float *__restrict__ row, float *u)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int p = q / sp.ncorner;
    int k = q - p * sp.ncorner;
    if (p >= sp.npoint) return;
    int64_t at = sp.base[p] + sp.corner_off[k];
    float w = sp.weight[(int64_t)p * 8 + k];
    atomicAdd(u + at, w * c[at] * row[p]);
}

// Zero-halo load along one axis.
__device__ __forceinline__ float ld0(const float *__restrict__ u, int64_t at, int64_t i,
                                     int64_t n)
{
    return (i >= 0 && i < n) ? u[at] : 0.0f;
}

// Laplacian at (i0, i1, i2): centre * u + sum_a sum_k coef[a][k] (u[-k] + u[+k]).
template <int M, bool THREE_D>
__device__ __forceinline__ float laplacian_at(const Geom &g, const Coef &cf,
                                              const float *__restrict__ u, int64_t at,
                                              int64_t i0, int64_t i1, int64_t i2)
{
    float lap = cf.centre * u[at];
#pragma unroll
    for (int k = 1; k <= M; k++) {
        float s2 = ld0(u, at - k, i2 - k, g.n[2]) + ld0(u, at + k, i2 + k, g.n[2]);
        float s1 = ld0(u, at - k * g.s1, i1 - k, g.n[1]) + ld0(u, at + k * g.s1, i1 + k, g.n[1]);
        lap = fmaf(cf.ax[2][k], s2, lap);
        lap = fmaf(cf.ax[1][k], s1, lap);
        if (THREE_D) {
            float s0 = ld0(u, at - k * g.s0, i0 - k, g.n[0]) + ld0(u, at + k * g.s0, i0 + k, g.n[0]);
            lap = fmaf(cf.ax[0][k], s0, lap);
        }
    }
    return lap;
}

// Acoustic leapfrog, in place over the previous slot:
//   u_prev <- 2u - u_prev + c L u - d (u - u_prev)
template <int M, bool THREE_D>
__global__ void acoustic_plain_kernel(Geom g, Coef cf, const float *__restrict__ u,
                                      const float *up, float *out, const float *__restrict__ c,
                                      const float *__restrict__ d)
{
    int64_t i2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i1 = blockIdx.y;
    if (i2 >= g.n[2]) return;
    for (int64_t i0 = 0; i0 < g.n[0]; i0++) {
        int64_t at = i0 * g.s0 + i1 * g.s1 + i2;
        float lap = laplacian_at<M, THREE_D>(g, cf, u, at, i0, i1, i2);
        float uc = u[at];
        float upv = up[at];
        // three explicit FMAs (2u is exact), the chain the tiled kernels use
        out[at] = fmaf(-d[at], uc - upv, fmaf(c[at], lap, fmaf(2.0f, uc, -upv)));
    }
}

// The imaging condition of K consecutive adjoint steps in one pass: for
// j = 0 .. K-1 in turn, grad += scale * mu[j] * (u[j] - 2 u[j+1] + u[j+2]),
// with mu[j] the adjoint state of time n - j and u[i] the forward state of
// time n - i.  Each forward state and grad are read once for the K steps
// (4 (2K + 4) bytes per point instead of 24 K); every step's FMA chain is
// imaging_kernel's, in its order, so the result equals K imaging_kernel
// launches (steps n, n-1, ...) bit for bit.
struct ImagingSteps {
    const float *mu[4];
    const float *u[6];
};

template <int K>
__global__ void imaging_steps_kernel(Geom g, float scale, ImagingSteps p, float *__restrict__ grad)
{
    const int64_t rows = g.n[0] * g.n[1];
    const int64_t groups = (g.n[2] + 3) / 4;  // float4 groups per row
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows * groups;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / groups;
        const int64_t c0 = 4 * (q - row * groups);
        const int64_t i0 = row / g.n[1];
        const int64_t i1 = row - i0 * g.n[1];
        const int64_t at = i0 * g.s0 + i1 * g.s1 + c0;
        if (c0 + 4 <= g.n[2]) {
            float4 u[K + 2];
#pragma unroll
            for (int i = 0; i < K + 2; i++) u[i] = *reinterpret_cast<const float4 *>(p.u[i] + at);
            float4 gr = *reinterpret_cast<const float4 *>(grad + at);
#pragma unroll
            for (int j = 0; j < K; j++) {
                const float4 m4 = *reinterpret_cast<const float4 *>(p.mu[j] + at);
                const float4 a = u[j], b = u[j + 1], e = u[j + 2];
                gr.x = fmaf(scale * m4.x, fmaf(-2.0f, b.x, a.x) + e.x, gr.x);
                gr.y = fmaf(scale * m4.y, fmaf(-2.0f, b.y, a.y) + e.y, gr.y);
                gr.z = fmaf(scale * m4.z, fmaf(-2.0f, b.z, a.z) + e.z, gr.z);
                gr.w = fmaf(scale * m4.w, fmaf(-2.0f, b.w, a.w) + e.w, gr.w);
            }
            *reinterpret_cast<float4 *>(grad + at) = gr;
        } else {
            for (int64_t k = 0; c0 + k < g.n[2]; k++) {
                const int64_t i = at + k;
                float t = grad[i];
#pragma unroll
                for (int j = 0; j < K; j++)
                    t = fmaf(scale * p.mu[j][i], fmaf(-2.0f, p.u[j + 1][i], p.u[j][i]) + p.u[j + 2][i], t);
                grad[i] = t;
            }
        }
    }
}

// grad += scale * mu * (u0 - 2 u1 + u2) over the interior: the imaging
// condition of the adjoint-state gradient with respect to m.
__global__ void imaging_kernel(Geom g, float scale, const float *__restrict__ mu,
                               const float *__restrict__ u0, const float *__restrict__ u1,
                               const float *__restrict__ u2, float *__restrict__ grad)
{
    const int64_t rows = g.n[0] * g.n[1];
    const int64_t groups = (g.n[2] + 3) / 4;  // float4 groups per row
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows * groups;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = q / groups;
        const int64_t c0 = 4 * (q - row * groups);
        const int64_t i0 = row / g.n[1];
        const int64_t i1 = row - i0 * g.n[1];
        const int64_t at = i0 * g.s0 + i1 * g.s1 + c0;
        if (c0 + 4 <= g.n[2]) {
            const float4 m4 = *reinterpret_cast<const float4 *>(mu + at);
            const float4 a = *reinterpret_cast<const float4 *>(u0 + at);
            const float4 b = *reinterpret_cast<const float4 *>(u1 + at);
            const float4 e = *reinterpret_cast<const float4 *>(u2 + at);
            float4 gr = *reinterpret_cast<const float4 *>(grad + at);
            // explicit FMAs, the order of the imaging fused into the tiled
            // adjoint step, so that the two agree bit for bit
            gr.x = fmaf(scale * m4.x, fmaf(-2.0f, b.x, a.x) + e.x, gr.x);
            gr.y = fmaf(scale * m4.y, fmaf(-2.0f, b.y, a.y) + e.y, gr.y);
            gr.z = fmaf(scale * m4.z, fmaf(-2.0f, b.z, a.z) + e.z, gr.z);
            gr.w = fmaf(scale * m4.w, fmaf(-2.0f, b.w, a.w) + e.w, gr.w);
            *reinterpret_cast<float4 *>(grad + at) = gr;
        } else {
            for (int64_t k = 0; c0 + k < g.n[2]; k++)
                grad[at + k] = fmaf(scale * mu[at + k], fmaf(-2.0f, u1[at + k], u0[at + k]) + u2[at + k], grad[at + k]);
        }
    }
}

// Explicit Euler diffusion: u_out <- u + a dt L u
template <int M, bool THREE_D>
__global__ void diffusion_plain_kernel(Geom g, Coef cf, float adt, const float *__restrict__ u,
                                       float *__restrict__ out)
{
    int64_t i2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t i1 = blockIdx.y;
    if (i2 >= g.n[2]) return;
    for (int64_t i0 = 0; i0 < g.n[0]; i0++) {
        int64_t at = i0 * g.s0 + i1 * g.s1 + i2;
        float lap = laplacian_at<M, THREE_D>(g, cf, u, at, i0, i1, i2);
        out[at] = fmaf(adt, lap, u[at]);
    }
}

// Linear Convection (Eq. 2dconvdiscr) on a 2D grid (rows d1 = x, columns
// d2 = y): first-order upwind, zero halo.  One thread per point.
__global__ void convection_plain_kernel(Geom g, float nux, float nuy, const float *__restrict__ u,
                                        float *__restrict__ out)
{
    const int64_t i2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i1 = blockIdx.y;
    if (i2 >= g.n[2]) return;
    const int64_t at = i1 * g.s1 + i2;
    const float uc = u[at];
    const float ux = i1 > 0 ? u[at - g.s1] : 0.0f;
    const float uy = i2 > 0 ? u[at - 1] : 0.0f;
    // two explicit FMAs, in the order the cluster kernel uses, so that both
    // paths give the same bits
    out[at] = fmaf(-nuy, uc - uy, fmaf(-nux, uc - ux, uc));
}

__device__ __forceinline__ void add_block_sum(double v, double *sum)
{
    __shared__ double part[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); i++) t += part[i];
        atomicAdd(sum, t);
    }
}

// Laplace equation (Eq. 2dlaplace_discr) Jacobi sweep with the boundary
// expressions: rows 0 and n1-1 keep their values (Dirichlet), then columns 0
// and n2-1 copy columns 1 and n2-2 (Neumann, corners included).
__global__ void jacobi_plain_kernel(Geom g, float wr, float wc, const float *__restrict__ p,
                                    float *__restrict__ out, double *sum)
{
    const int64_t i2 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i1 = blockIdx.y;
    float v = 0.0f;
    if (i2 < g.n[2]) {
        const int64_t cc = i2 == 0 ? 1 : (i2 == g.n[2] - 1 ? g.n[2] - 2 : i2);
        const int64_t q = i1 * g.s1 + cc;
        if (i1 == 0 || i1 == g.n[1] - 1)
            v = p[q];
        else
            v = wr * (p[q - g.s1] + p[q + g.s1]) + wc * (p[q - 1] + p[q + 1]);
        out[i1 * g.s1 + i2] = v;
    }
    if (sum) add_block_sum(fabs((double)v), sum);
}

__global__ void abs_sum_kernel(Geom g, const float *__restrict__ u, double *sum)
{
    double t = 0.0;
    const int64_t total = g.n[0] * g.n[1] * g.n[2];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i2 = q % g.n[2], r = q / g.n[2];
        const int64_t i1 = r % g.n[1], i0 = r / g.n[1];
        t += fabs((double)u[i0 * g.s0 + i1 * g.s1 + i2]);
    }
    add_block_sum(t, sum);
}

int grid_stride_blocks(int64_t total)
{
    int64_t b = (total + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_coefficients(const Geom &g, const float *m, const float *eta, double dt,
                                float *c, float *d, cudaStream_t st)
{
    int64_t total = g.n[0] * g.n[1] * g.n[2];
    coefficients_kernel<<<grid_stride_blocks(total), kThreads, 0, st>>>(
        g, m, eta, (float)(dt * dt), (float)dt, c, d);
    return cudaGetLastError();
}

cudaError_t launch_min_reduce(const Geom &g, const float *m, unsigned int *out_bits,
                              cudaStream_t st)
{
    int64_t total = g.n[0] * g.n[1] * g.n[2];
    min_reduce_kernel<<<grid_stride_blocks(total), kThreads, 0, st>>>(g, m, out_bits);
    return cudaGetLastError();
}

cudaError_t prepare_interpolate()
{
    cudaFuncAttributes attr;
    return cudaFuncGetAttributes(&attr, interpolate_kernel);
}

cudaError_t launch_interpolate(const SparseDev &sp, const float *u, float *out_row,
                               cudaStream_t st)
{
    if (sp.npoint <= 0) return cudaSuccess;
    interpolate_kernel<<<(sp.npoint + 127) / 128, 128, 0, st>>>(sp, u, out_row);
    return cudaGetLastError();
}

cudaError_t launch_inject(const SparseDev &sp, const float *c, const float *row, float *u,
                          cudaStream_t st)
{
    if (sp.npoint <= 0) return cudaSuccess;
    int total = sp.npoint * sp.ncorner;
    inject_kernel<<<(total + 127) / 128, 128, 0, st>>>(sp, c, row, u);
    return cudaGetLastError();
}

#define FD_FOR_EACH_M(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

cudaError_t launch_imaging(const Geom &g, float scale, const float *mu, const float *u0, const float *u1,
                           const float *u2, float *grad, cudaStream_t st)
{
    int64_t total = g.n[0] * g.n[1] * ((g.n[2] + 3) / 4);
    imaging_kernel<<<grid_stride_blocks(total), kThreads, 0, st>>>(g, scale, mu, u0, u1, u2, grad);
    return cudaGetLastError();
}

cudaError_t launch_imaging_steps(const Geom &g, float scale, int k, const float *const *mu, const float *const *u,
                                 float *grad, cudaStream_t st)
{
    if (k < 1 || k > 4) return cudaErrorInvalidValue;
    ImagingSteps p{};
    for (int j = 0; j < k; j++) p.mu[j] = mu[j];
    for (int i = 0; i < k + 2; i++) p.u[i] = u[i];
    const int64_t total = g.n[0] * g.n[1] * ((g.n[2] + 3) / 4);
    const int blocks = grid_stride_blocks(total);
    switch (k) {
    case 1: imaging_steps_kernel<1><<<blocks, kThreads, 0, st>>>(g, scale, p, grad); break;
    case 2: imaging_steps_kernel<2><<<blocks, kThreads, 0, st>>>(g, scale, p, grad); break;
    case 3: imaging_steps_kernel<3><<<blocks, kThreads, 0, st>>>(g, scale, p, grad); break;
    default: imaging_steps_kernel<4><<<blocks, kThreads, 0, st>>>(g, scale, p, grad); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_acoustic_plain(int M, const Geom &g, const Coef &cf, const float *u,
                                  const float *up, float *out, const float *c, const float *d, cudaStream_t st)
{
    dim3 grid((unsigned)((g.n[2] + 127) / 128), (unsigned)g.n[1]);
    bool three = g.ndim == 3;
    switch (M) {
#define CASE(MM)                                                                          \
    case MM:                                                                              \
        if (three)                                                                        \
            acoustic_plain_kernel<MM, true><<<grid, 128, 0, st>>>(g, cf, u, up, out, c, d);  \
        else                                                                                \
            acoustic_plain_kernel<MM, false><<<grid, 128, 0, st>>>(g, cf, u, up, out, c, d); \
        break;
        FD_FOR_EACH_M(CASE)
#undef CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_diffusion_plain(int M, const Geom &g, const Coef &cf, float adt,
                                   const float *u, float *out, cudaStream_t st)
{
    dim3 grid((unsigned)((g.n[2] + 127) / 128), (unsigned)g.n[1]);
    bool three = g.ndim == 3;
    switch (M) {
#define CASE(MM)                                                                          \
    case MM:                                                                              \
        if (three)                                                                        \
            diffusion_plain_kernel<MM, true><<<grid, 128, 0, st>>>(g, cf, adt, u, out);   \
        else                                                                              \
            diffusion_plain_kernel<MM, false><<<grid, 128, 0, st>>>(g, cf, adt, u, out);  \
        break;
        FD_FOR_EACH_M(CASE)
#undef CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_convection_plain(const Geom &g, float nux, float nuy, const float *u, float *out,
                                    cudaStream_t st)
{
    dim3 grid((unsigned)((g.n[2] + 127) / 128), (unsigned)g.n[1]);
    convection_plain_kernel<<<grid, 128, 0, st>>>(g, nux, nuy, u, out);
    return cudaGetLastError();
}

cudaError_t launch_jacobi_plain(const Geom &g, float wr, float wc, const float *p, float *out, double *sum,
                                cudaStream_t st)
{
    dim3 grid((unsigned)((g.n[2] + 127) / 128), (unsigned)g.n[1]);
    jacobi_plain_kernel<<<grid, 128, 0, st>>>(g, wr, wc, p, out, sum);
    return cudaGetLastError();
}

cudaError_t launch_abs_sum(const Geom &g, const float *u, double *sum, cudaStream_t st)
{
    abs_sum_kernel<<<grid_stride_blocks(g.n[0] * g.n[1] * g.n[2]), kThreads, 0, st>>>(g, u, sum);
    return cudaGetLastError();
}

}  // namespace fdgb
