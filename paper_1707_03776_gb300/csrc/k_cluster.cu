// Explicit diffusion on small 2D grids: the whole time loop in one launch of
// one thread-block cluster.
//
// A 2D grid that fits in the shared memory of a cluster (the 254^2 interior of
// the 256^2 ring workload needs 2 x 34 x 264 floats per CTA with 8 CTAs) is
// split into row strips, one per CTA.  Each CTA keeps its strip plus M halo
// rows above and below, twice (ping-pong), in shared memory.  Per step every
// thread updates its points from one buffer into the other and, for the M
// first and last rows of the strip, also writes the new values into the
// neighbouring CTAs' halo rows through distributed shared memory; one cluster
// barrier then separates the steps.  Grid data touches global memory only at
// the start (u^{t0}) and at the end (the last two states, so that the slot
// convention of per-step launches holds: slot n%2 holds u^n).
#include <cooperative_groups.h>

#include "fd_internal.h"
#include "fd_internal_host.h"

namespace cg = cooperative_groups;

namespace fdgb {

namespace {

constexpr int kClusterThreads = 512;

struct ClusterArgs {
    int rows;         // grid rows (axis d1 of the 3-axis view)
    int cols;         // grid columns (contiguous axis)
    long long s1;     // row stride in global memory (elements)
    int strip;        // rows per CTA at most
    int width;        // shared row pitch: cols + 2M, rounded to 4
    int nclusters;    // CTAs in the cluster
};

template <int M>
__global__ void __launch_bounds__(kClusterThreads, 1)
    diffusion_cluster_kernel(const ClusterArgs a, const Coef cf, float adt, const float *__restrict__ u0,
                             float *__restrict__ out_last, float *__restrict__ out_prev, int nt)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ __align__(16) float sbuf[];
    const int W = a.width;
    const int H = a.strip + 2 * M;  // rows held: halo + strip + halo
    float *const buf0 = sbuf;
    float *const buf1 = sbuf + H * W;

    const int r0 = (int)((long long)rank * a.rows / a.nclusters);
    const int r1 = (int)((long long)(rank + 1) * a.rows / a.nclusters);
    const int nr = r1 - r0;
    const int tid = threadIdx.x;

    // load rows r0-M .. r1+M-1 (zero outside the grid) and zero the side halos
    for (int q = tid; q < 2 * H * W; q += blockDim.x) {
        const int b = q / (H * W);
        const int rem = q - b * H * W;
        const int lr = rem / W;
        const int c = rem - lr * W - M;
        const int gr = r0 - M + lr;
        float v = 0.0f;
        if (b == 0 && c >= 0 && c < a.cols && gr >= 0 && gr < a.rows && lr < nr + 2 * M)
            v = u0[(long long)gr * a.s1 + c];
        (b == 0 ? buf0 : buf1)[rem] = v;
    }
    cluster.sync();

    float *up_nb = nullptr;  // neighbour above (rank-1): its bottom halo rows
    float *dn_nb = nullptr;  // neighbour below (rank+1): its top halo rows
    const int npts = nr * a.cols;
    for (int step = 0; step < nt; step++) {
        const float *src = (step & 1) ? buf1 : buf0;
        float *dst = (step & 1) ? buf0 : buf1;
        if (rank > 0) up_nb = cluster.map_shared_rank(dst, rank - 1);
        if (rank + 1 < a.nclusters) dn_nb = cluster.map_shared_rank(dst, rank + 1);
        for (int p = tid; p < npts; p += blockDim.x) {
            const int lr = p / a.cols;
            const int c = p - lr * a.cols;
            const int at = (lr + M) * W + c + M;
            float lap = cf.centre * src[at];
#pragma unroll
            for (int k = 1; k <= M; k++) {
                lap = fmaf(cf.ax[2][k], src[at - k] + src[at + k], lap);
                lap = fmaf(cf.ax[1][k], src[at - k * W] + src[at + k * W], lap);
            }
            const float v = fmaf(adt, lap, src[at]);
            dst[at] = v;
            // the neighbour above holds our first M rows as its last M halo rows
            if (lr < M && up_nb) {
                const int nb_nr = r0 - (int)((long long)(rank - 1) * a.rows / a.nclusters);
                up_nb[(nb_nr + M + lr) * W + c + M] = v;
            }
            if (lr >= nr - M && dn_nb) dn_nb[(lr - (nr - M)) * W + c + M] = v;
        }
        cluster.sync();
    }

    // the last state (step nt) and the one before it (step nt-1, or u^{t0}
    // when nt == 1 -- the caller then skips out_prev)
    for (int p = tid; p < npts; p += blockDim.x) {
        const int lr = p / a.cols;
        const int c = p - lr * a.cols;
        const int at = (lr + M) * W + c + M;
        const long long g = (long long)(r0 + lr) * a.s1 + c;
        out_last[g] = ((nt & 1) ? buf1 : buf0)[at];
        if (out_prev) out_prev[g] = ((nt & 1) ? buf0 : buf1)[at];
    }
}

template <int M>
cudaError_t launch_cluster_m(const ClusterArgs &a, const Coef &cf, float adt, const float *u0, float *out_last,
                             float *out_prev, int nt, size_t smem, cudaStream_t st)
{
    auto kern = diffusion_cluster_kernel<M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a.nclusters > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.nclusters);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.nclusters;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, cf, adt, u0, out_last, out_prev, nt);
}

}  // namespace

bool diffusion_cluster_fits(int M, const Geom &g, int *nclusters, size_t *smem_out)
{
    if (g.ndim != 2 || g.n[0] != 1 || M < 1 || M > kMaxHalfWidth) return false;
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    const int rows = (int)g.n[1], cols = (int)g.n[2];
    const int width = (cols + 2 * M + 3) / 4 * 4;
    for (int c : {8, 16}) {
        const int strip = (rows + c - 1) / c;
        if (rows / c < M) continue;  // every strip must cover its neighbours' halo
        const size_t smem = sizeof(float) * 2 * (size_t)(strip + 2 * M) * width;
        if (smem <= (size_t)smem_max) {
            *nclusters = c;
            *smem_out = smem;
            return true;
        }
    }
    return false;
}

cudaError_t launch_diffusion_cluster(int M, const Geom &g, const Coef &cf, float adt, const float *u0,
                                     float *out_last, float *out_prev, int nt, int nclusters, size_t smem,
                                     cudaStream_t st)
{
    ClusterArgs a;
    a.rows = (int)g.n[1];
    a.cols = (int)g.n[2];
    a.s1 = g.s1;
    a.nclusters = nclusters;
    a.strip = (a.rows + nclusters - 1) / nclusters;
    a.width = (a.cols + 2 * M + 3) / 4 * 4;
    switch (M) {
#define CASE(MM) \
    case MM: return launch_cluster_m<MM>(a, cf, adt, u0, out_last, out_prev, nt, smem, st);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdgb
