// Small 2D grids: the whole time loop (or convergence loop) in one launch of
// one thread-block cluster, with K steps between halo exchanges.
//
// The grid's rows are split into strips, one per CTA.  Each CTA keeps its
// strip plus H = K*M halo rows above and below, twice (ping-pong), in shared
// memory.  A block of K steps runs without any inter-CTA communication: step
// j of the block also updates the (K-1-j)*M halo rows nearest the strip
// (redundantly with the neighbour, same arithmetic), so the rows the next step
// reads are always current.  After the block every CTA writes its first and
// last H rows into its neighbours' inboxes through distributed shared memory,
// one cluster barrier separates the writes from the reads, and each CTA copies
// its inbox into its halo rows.  Inboxes alternate between two buffers by
// block parity, so one barrier per block is enough (a neighbour can only write
// the same inbox again after the next barrier, which this CTA reaches after
// reading it).  Temporal blocking trades (K-1)*M redundant rows per strip for
// K-times fewer cluster barriers.
//
// Update rules (the operator kinds of the 2D examples):
//   diffusion  u+ = u + a dt L u            (SO 2..16, zero halo)
//   upwind     u+ = u - nu_x (u - u[i-1,j]) - nu_y (u - u[i,j-1])
//              (Linear Convection, Eq. 2dconvdiscr; zero halo)
//   jacobi     Laplace equation, Eq. 2dlaplace_discr, on interior nodes; the
//              first and last rows keep their values (Dirichlet), then the
//              first and last columns copy their neighbour column (Neumann,
//              corners included) -- in the order the paper lists them.
// The jacobi rule can stop on the L1 criterion r = |S+ - S| / S < tol, with S
// the grid's sum of |p|: every CTA adds its rows' partial sum (compensated
// FP32, ~48 significant bits) to a slot of its shared memory, and after the
// barrier thread 0 of every CTA adds all slots in rank order in FP64, so all
// take the same decision.
//
// Grid data touches global memory only at the start (u^{t0}) and at the end:
// the last state goes to slot (t0+steps)%2 and the one before it to the other
// slot, which keeps the convention of per-step launches (slot n%2 holds u^n).
#include <cooperative_groups.h>

#include <algorithm>

#include "fd_internal.h"
#include "fd_internal_host.h"

namespace cg = cooperative_groups;

namespace fdgb {

namespace {

constexpr int kCThreads = 512;

struct ClusterArgs {
    int rows, cols;   // grid rows (axis d1) and columns (contiguous axis d2)
    long long s1;     // row stride in global memory (elements)
    int strip;        // rows per CTA at most
    int width;        // shared row pitch: cols + 2 hc, rounded to 4
    int hc;           // zero columns on each side
    int halo;         // halo rows on each side: K*M (M when alone)
    int K;            // steps between exchanges
    int nctas;        // CTAs in the cluster
    int tc, tr;       // threads along columns (float4 chunks when vec) and rows
    int vec;          // SO2 diffusion: each thread updates 4 columns with 128-bit loads
};

struct RuleArgs {
    Coef cf;
    float adt;        // diffusion: a dt
    float nux, nuy;   // upwind: c dt / h per axis
    float wr, wc;     // jacobi: weights of the row and column neighbours
};

template <int RULE, int M>
__device__ __forceinline__ float apply_rule(const float *__restrict__ src, int at, int W, int gr, int c,
                                            const ClusterArgs &a, const RuleArgs &ra)
{
    if (RULE == kRuleDiffusion) {
        const float u = src[at];
        float lap = ra.cf.centre * u;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            lap = fmaf(ra.cf.ax[2][k], src[at - k] + src[at + k], lap);
            lap = fmaf(ra.cf.ax[1][k], src[at - k * W] + src[at + k * W], lap);
        }
        return fmaf(ra.adt, lap, u);
    } else if (RULE == kRuleUpwind) {
        const float u = src[at];
        // u - nux (u - u_up) - nuy (u - u_left), as two explicit FMAs so that
        // the packed 4-column sweep can repeat it bit for bit
        return fmaf(-ra.nuy, u - src[at - 1], fmaf(-ra.nux, u - src[at - W], u));
    } else {
        const int cc = c == 0 ? 1 : (c == a.cols - 1 ? a.cols - 2 : c);
        const int q = at + (cc - c);
        if (gr == 0 || gr == a.rows - 1) return src[q];
        return ra.wr * (src[q - W] + src[q + W]) + ra.wc * (src[q - 1] + src[q + 1]);
    }
}

// Compensated FP32 sum (hi + lo carries ~48 significant bits): Knuth's
// TwoSum of the high parts, the rounding error folded into the low part.
// FP64 arithmetic is slow on this GPU; the convergence sums only need ~1e-12.
__device__ __forceinline__ void sum2_add(float &hi, float &lo, float bhi, float blo)
{
    const float s = hi + bhi;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (bhi - bp);
    lo = lo + blo + e;
    hi = s;
}

// Block-wide compensated sum; the result (as FP64) is valid in thread 0.
__device__ __forceinline__ double block_sum2(float hi, float lo, float *scratch)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        sum2_add(hi, lo, oh, ol);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        scratch[2 * w] = hi;
        scratch[2 * w + 1] = lo;
    }
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        // second stage in warp 0: its lanes take the warps' pairs
        const int nw = (int)(blockDim.x >> 5);
        hi = l < nw ? scratch[2 * l] : 0.0f;
        lo = l < nw ? scratch[2 * l + 1] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
            const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
            sum2_add(hi, lo, oh, ol);
        }
        if (l == 0) t = (double)hi + (double)lo;
    }
    __syncthreads();
    return t;
}

// Block-wide compensated sum left in every thread: each warp reduces the
// warps' pairs itself after one barrier (the butterfly of exact TwoSum steps
// gives every lane the same bits).  scratch holds 64 floats.
__device__ __forceinline__ void block_sum2_all(float &hi, float &lo, float *scratch)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        sum2_add(hi, lo, oh, ol);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        scratch[2 * w] = hi;
        scratch[2 * w + 1] = lo;
    }
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    hi = l < nw ? scratch[2 * l] : 0.0f;
    lo = l < nw ? scratch[2 * l + 1] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
        sum2_add(hi, lo, oh, ol);
    }
}

// |a - b| < t * b for double-float a = (ah, al), b = (bh, bl) > 0 and
// t = (th, tl): the difference and the product carried to ~48 bits (TwoSum,
// and TwoProd with fmaf), then compared as double-float numbers.
__device__ __forceinline__ bool df_rel_below(float ah, float al, float bh, float bl, float th, float tl)
{
    float dh = ah - bh;
    const float bp = dh - ah;
    float dl = ((ah - (dh - bp)) + (-bh - bp)) + (al - bl);
    const float s = dh + dl;  // renormalise the difference
    dl = dl - (s - dh);
    dh = s;
    if (dh < 0.0f) {
        dh = -dh;
        dl = -dl;
    }
    const float ph = th * bh;
    const float pl = fmaf(th, bh, -ph) + (th * bl + tl * bh);
    const float q = ph + pl;
    const float ql = pl - (q - ph);
    return dh < q || (dh == q && dl < ql);
}

template <int RULE, int M>
__global__ void __launch_bounds__(kCThreads, 1)
    cluster_stencil_kernel(const ClusterArgs a, const RuleArgs ra, const float *__restrict__ u0, float *slot0,
                           float *slot1, long long t0, long long nt, double tol, long long *res_steps,
                           double *res_r)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ __align__(16) unsigned char craw[];
    const int W = a.width, H = a.halo;
    const int HR = a.strip + 2 * H;  // rows held
    float *buf[2];
    buf[0] = reinterpret_cast<float *>(craw);
    buf[1] = buf[0] + HR * W;
    float *inbox = buf[1] + HR * W;                        // [2 parities][2 sides][H][cols]
    double *part = reinterpret_cast<double *>(inbox + 4 * H * a.cols);  // [2] partial sums
    float *scratch = reinterpret_cast<float *>(part + 2);  // [2 parities][32 warps][hi, lo]
    volatile int *flag = reinterpret_cast<volatile int *>(scratch + 128);

    const int r0 = (int)((long long)rank * a.rows / a.nctas);
    const int r1 = (int)((long long)(rank + 1) * a.rows / a.nctas);
    const int nr = r1 - r0;
    const int tid = threadIdx.x;
    const int tc = tid % a.tc, tr = tid / a.tc;
    const bool lane_on = tr < a.tr;
    const bool converge = RULE == kRuleJacobi && tol > 0.0;
    // a cluster of one CTA needs only block barriers and its own shared memory
    const bool alone = a.nctas == 1;
    auto barrier = [&]() {
        if (alone)
            __syncthreads();
        else
            cluster.sync();
    };
    auto part_of = [&](int k, int slot) -> double {
        return alone ? part[slot] : *cluster.map_shared_rank(&part[slot], k);
    };

    // rows r0-H .. r1+H-1 of u^{t0} (zero outside the grid) into buf[0];
    // buf[1] zero, so that rows outside the grid and the side columns stay 0
    float sh = 0.0f, sl = 0.0f;
    for (int q = tid; q < HR * W; q += blockDim.x) {
        const int lr = q / W;
        const int c = q - lr * W - a.hc;
        const int gr = r0 - H + lr;
        float v = 0.0f;
        if (c >= 0 && c < a.cols && gr >= 0 && gr < a.rows && lr < nr + 2 * H) v = u0[(long long)gr * a.s1 + c];
        buf[0][q] = v;
        buf[1][q] = 0.0f;
        if (converge && gr >= r0 && gr < r1 && c >= 0 && c < a.cols) sum2_add(sh, sl, fabsf(v), 0.0f);
    }
    int cur = 0, par = 0;
    long long done = 0;
    double r_last = INFINITY;
    bool stop = false;
    if (RULE == kRuleJacobi && converge && alone) {
        // One CTA to convergence: one barrier per sweep.  Every thread holds
        // S^n as a double-float pair and takes the same decision from the
        // same bits, so no flag and no FP64 arithmetic are needed in the loop.
        float oh = sh, ol = sl;
        block_sum2_all(oh, ol, scratch);
        par = 1;  // the first sweep's partials go to the other scratch half
        const float th = (float)tol, tl = (float)(tol - (double)th);
        float dh = 0.0f, dl = 0.0f, ph = 0.0f, pl = 0.0f;
        while (done < nt) {
            sh = sl = 0.0f;
            const float *src = buf[cur];
            float *dst = buf[cur ^ 1];
            if (lane_on)
                for (int lr = tr; lr < nr; lr += a.tr) {
                    const int base = (lr + H) * W + a.hc;
                    for (int c = tc; c < a.cols; c += a.tc) {
                        const float v = apply_rule<RULE, M>(src, base + c, W, lr, c, a, ra);
                        dst[base + c] = v;
                        sum2_add(sh, sl, fabsf(v), 0.0f);
                    }
                }
            cur ^= 1;
            done++;
            // the barrier inside also orders this sweep's writes before the
            // next sweep's reads; the scratch halves alternate by parity
            block_sum2_all(sh, sl, scratch + 64 * par);
            par ^= 1;
            const bool hit = oh > 0.0f && df_rel_below(sh, sl, oh, ol, th, tl);
            ph = oh;
            pl = ol;
            dh = sh;
            dl = sl;
            oh = sh;
            ol = sl;
            if (hit) break;
        }
        if (done > 0 && ph > 0.0f) {
            const double sn = (double)dh + (double)dl, so = (double)ph + (double)pl;
            r_last = fabs(sn - so) / so;
        }
        stop = true;
    }
    // the convergence state lives in thread 0 of every CTA (all take the same
    // decision from the same partial sums) and reaches the others by `flag`
    double s_old = 0.0;
    if (converge && !stop) {
        const double t = block_sum2(sh, sl, scratch);
        if (tid == 0) part[1] = t;
    }
    if (!stop) barrier();
    if (converge && !stop && tid == 0)
        for (int k = 0; k < a.nctas; k++) s_old += part_of(k, 1);

    while (done < nt && !stop) {
        // the L1 criterion is taken after every sweep: blocks of one step
        const int Kb = converge ? 1 : (int)((nt - done) < (long long)a.K ? (nt - done) : (long long)a.K);
        sh = sl = 0.0f;
        for (int j = 0; j < Kb; j++) {
            const int ext = (Kb - 1 - j) * M;
            const int lo = max(-ext, -r0), hi = min(nr + ext, a.rows - r0);
            const float *src = buf[cur];
            float *dst = buf[cur ^ 1];
            if ((RULE == kRuleDiffusion || RULE == kRuleUpwind) && M == 1 && a.vec) {
                // 4 columns per thread: rows padded with 4 zero columns so
                // every chunk is 16-byte aligned; the left and right
                // neighbours come from the adjacent chunks (same arithmetic
                // per point as apply_rule)
                if (lane_on)
                    for (int lr = lo + tr; lr < hi; lr += a.tr) {
                        const int base = (lr + H) * W + a.hc;
                        for (int c = 4 * tc; c < a.cols; c += 4 * a.tc) {
                            const float *p = src + base + c;
                            const float4 cu = *reinterpret_cast<const float4 *>(p);
                            const float4 lf = *reinterpret_cast<const float4 *>(p - 4);
                            const float4 rt = *reinterpret_cast<const float4 *>(p + 4);
                            const float4 up = *reinterpret_cast<const float4 *>(p - W);
                            const float4 dn = *reinterpret_cast<const float4 *>(p + W);
                            const float uu[6] = {lf.w, cu.x, cu.y, cu.z, cu.w, rt.x};
                            // the 4 points as two pairs on the packed FP32
                            // instructions, each lane in the scalar order of
                            // apply_rule (bitwise the same results)
                            float o[4];
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const float2 u2 = h ? make_float2(cu.z, cu.w) : make_float2(cu.x, cu.y);
                                const float2 up2 = h ? make_float2(up.z, up.w) : make_float2(up.x, up.y);
                                float2 r2;
                                if (RULE == kRuleDiffusion) {
                                    const float2 dn2 = h ? make_float2(dn.z, dn.w) : make_float2(dn.x, dn.y);
                                    // left + right straddles a 64-bit register pair: scalar adds
                                    const float2 s2 = make_float2(uu[2 * h] + uu[2 * h + 2], uu[2 * h + 1] + uu[2 * h + 3]);
                                    float2 lap = __fmul2_rn(make_float2(ra.cf.centre, ra.cf.centre), u2);
                                    lap = __ffma2_rn(make_float2(ra.cf.ax[2][1], ra.cf.ax[2][1]), s2, lap);
                                    lap = __ffma2_rn(make_float2(ra.cf.ax[1][1], ra.cf.ax[1][1]), __fadd2_rn(up2, dn2), lap);
                                    r2 = __ffma2_rn(make_float2(ra.adt, ra.adt), lap, u2);
                                } else {
                                    // the two FMAs of apply_rule's upwind form; x - y
                                    // is x + (-y) exactly
                                    const float2 lf2 = make_float2(uu[2 * h], uu[2 * h + 1]);
                                    const float2 dx = __fadd2_rn(u2, make_float2(-up2.x, -up2.y));
                                    const float2 dy = __fadd2_rn(u2, make_float2(-lf2.x, -lf2.y));
                                    const float2 a = __ffma2_rn(make_float2(-ra.nux, -ra.nux), dx, u2);
                                    r2 = __ffma2_rn(make_float2(-ra.nuy, -ra.nuy), dy, a);
                                }
                                o[2 * h] = r2.x;
                                o[2 * h + 1] = r2.y;
                            }
                            float *d = dst + base + c;
                            if (c + 3 < a.cols) {
                                *reinterpret_cast<float4 *>(d) = make_float4(o[0], o[1], o[2], o[3]);
                            } else {
                                // the zero columns past the grid must stay zero
#pragma unroll
                                for (int i = 0; i < 4; i++)
                                    if (c + i < a.cols) d[i] = o[i];
                            }
                        }
                    }
            } else if (lane_on) {
                for (int lr = lo + tr; lr < hi; lr += a.tr) {
                    const int base = (lr + H) * W + a.hc;
                    const int gr = r0 + lr;
                    for (int c = tc; c < a.cols; c += a.tc) {
                        const float v = apply_rule<RULE, M>(src, base + c, W, gr, c, a, ra);
                        dst[base + c] = v;
                        if (converge && lr >= 0 && lr < nr) sum2_add(sh, sl, fabsf(v), 0.0f);
                    }
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        done += Kb;
        if (converge) {
            const double t = block_sum2(sh, sl, scratch);
            if (tid == 0) part[par] = t;
        }
        // first H rows to the neighbour above (its bottom inbox), last H rows
        // to the neighbour below (its top inbox)
        const int nH = H * a.cols;
        if (a.nctas > 1 && (done < nt || converge)) {
            float *up = rank > 0 ? cluster.map_shared_rank(inbox, rank - 1) + (par * 2 + 1) * nH : nullptr;
            float *dn = rank + 1 < a.nctas ? cluster.map_shared_rank(inbox, rank + 1) + (par * 2 + 0) * nH : nullptr;
            const float *s = buf[cur];
            for (int q = tid; q < nH; q += blockDim.x) {
                const int lr = q / a.cols, c = q - lr * a.cols;
                if (up) up[q] = s[(lr + H) * W + a.hc + c];
                if (dn) dn[q] = s[(nr - H + lr + H) * W + a.hc + c];
            }
        }
        barrier();
        if (converge) {
            if (tid == 0) {
                double s_new = 0.0;
                for (int k = 0; k < a.nctas; k++) s_new += part_of(k, par);
                // r < tol as a product (FP64 division is slow here); r itself
                // is formed when the loop ends
                const bool hit = s_old > 0.0 && fabs(s_new - s_old) < tol * s_old;
                if (hit || done >= nt) r_last = s_old > 0.0 ? fabs(s_new - s_old) / s_old : INFINITY;
                *flag = hit ? 1 : 0;
                s_old = s_new;
            }
            __syncthreads();
            stop = *flag != 0;
        }
        if (a.nctas > 1 && done < nt && !stop) {
            float *d = buf[cur];
            const float *top = inbox + (par * 2 + 0) * nH, *bot = inbox + (par * 2 + 1) * nH;
            for (int q = tid; q < nH; q += blockDim.x) {
                const int lr = q / a.cols, c = q - lr * a.cols;
                if (rank > 0) d[lr * W + a.hc + c] = top[q];
                if (rank + 1 < a.nctas) d[(nr + H + lr) * W + a.hc + c] = bot[q];
            }
            __syncthreads();
        }
        par ^= 1;
    }

    // u^{t0+done} and u^{t0+done-1} into their slots
    if (done > 0) {
        float *last = ((t0 + done) & 1) ? slot1 : slot0;
        float *prev = ((t0 + done - 1) & 1) ? slot1 : slot0;
        for (int q = tid; q < nr * a.cols; q += blockDim.x) {
            const int lr = q / a.cols, c = q - lr * a.cols;
            const long long g = (long long)(r0 + lr) * a.s1 + c;
            const int at = (lr + H) * W + a.hc + c;
            last[g] = buf[cur][at];
            prev[g] = buf[cur ^ 1][at];
        }
    }
    if (rank == 0 && tid == 0 && res_steps) {
        *res_steps = done;
        *res_r = r_last;
    }
    // no CTA may leave while a neighbour can still read its shared memory
    barrier();
}

size_t cluster_smem_bytes(int strip, int halo, int width, int cols)
{
    // two buffers, the inboxes, 2 partial sums, 2 x 32 warps' (hi, lo), a flag
    return sizeof(float) * (2 * (size_t)(strip + 2 * halo) * width + 4 * (size_t)halo * cols) +
           sizeof(double) * 2 + sizeof(float) * 128 + 16;
}

template <int RULE, int M>
cudaError_t launch_rule(const ClusterPlan &p, const ClusterArgs &a, const RuleArgs &ra, const float *u0, float *s0,
                        float *s1, long long t0, long long nt, double tol, long long *res_steps, double *res_r,
                        cudaStream_t st)
{
    auto kern = cluster_stencil_kernel<RULE, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    if (a.nctas > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.nctas);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.nctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, ra, u0, s0, s1, t0, nt, tol, res_steps, res_r);
}

template <int RULE>
cudaError_t launch_m(int M, const ClusterPlan &p, const ClusterArgs &a, const RuleArgs &ra, const float *u0,
                     float *s0, float *s1, long long t0, long long nt, double tol, long long *rs, double *rr,
                     cudaStream_t st)
{
    if constexpr (RULE != kRuleDiffusion) {
        if (M != 1) return cudaErrorInvalidValue;
        return launch_rule<RULE, 1>(p, a, ra, u0, s0, s1, t0, nt, tol, rs, rr, st);
    } else {
        switch (M) {
#define CASE(MM) \
    case MM: return launch_rule<RULE, MM>(p, a, ra, u0, s0, s1, t0, nt, tol, rs, rr, st);
            CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        }
        return cudaErrorInvalidValue;
    }
}

// Whether a cluster of n CTAs with this shared memory can be resident (a
// 16-CTA cluster needs 16 free SMs of one GPC).
template <int RULE, int M>
bool clusters_fit(int n, size_t smem)
{
    auto kern = cluster_stencil_kernel<RULE, M>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    if (n > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)n;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int num = 0;
    if (cudaOccupancyMaxActiveClusters(&num, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return num >= 1;
}

bool clusters_fit_rule(int rule, int M, int n, size_t smem)
{
    if (rule == kRuleUpwind) return M == 1 && clusters_fit<kRuleUpwind, 1>(n, smem);
    if (rule == kRuleJacobi) return M == 1 && clusters_fit<kRuleJacobi, 1>(n, smem);
    switch (M) {
#define CASE(MM) \
    case MM: return clusters_fit<kRuleDiffusion, MM>(n, smem);
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    return false;
}

// SO2 diffusion and the upwind rule run the 4-column (float4) sweep
bool cluster_vec(int rule, int M) { return (rule == kRuleDiffusion || rule == kRuleUpwind) && M == 1; }

// zero columns on each side of a shared row, and the row pitch
int cluster_hc(int rule, int M) { return cluster_vec(rule, M) ? 4 : M; }
int cluster_width(int rule, int M, int cols) { return (cols + 2 * cluster_hc(rule, M) + 3) / 4 * 4; }

ClusterArgs make_args(const ClusterPlan &p, const Geom &g)
{
    ClusterArgs a;
    a.rows = (int)g.n[1];
    a.cols = (int)g.n[2];
    a.s1 = g.s1;
    a.nctas = p.nctas;
    a.strip = (a.rows + p.nctas - 1) / p.nctas;
    a.hc = cluster_hc(p.rule, p.M);
    a.width = cluster_width(p.rule, p.M, a.cols);
    a.K = p.K;
    a.halo = p.halo;
    a.vec = cluster_vec(p.rule, p.M) ? 1 : 0;
    const int units = a.vec ? (a.cols + 3) / 4 : a.cols;  // work items along a row
    a.tc = std::min(kCThreads, (units + 31) / 32 * 32);
    a.tr = kCThreads / a.tc;
    return a;
}

}  // namespace

// Pick the cluster size and the steps per exchange of a rule on a 2D grid:
// the fewest CTAs that keep at most ~8 points per thread and step (tiny grids
// stay in one CTA, where a block barrier is cheaper than a cluster one), else
// the most that fit; K = `want_k` if > 0, else 1 + strip/(4M) (at most ~25 %
// redundant rows), capped at 8 and so that every strip covers the halo.
bool cluster_plan_build(int rule, int M, const Geom &g, int want_k, ClusterPlan *out)
{
    out->ok = false;
    if (g.ndim != 2 || g.n[0] != 1 || M < 1 || M > kMaxHalfWidth) return false;
    if (rule != kRuleDiffusion && M != 1) return false;
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    const int rows = (int)g.n[1], cols = (int)g.n[2];
    if (rows < 1 || cols < 1 || (rule == kRuleJacobi && (rows < 3 || cols < 3))) return false;
    const int width = cluster_width(rule, M, cols);
    const long long pts = (long long)rows * cols;
    int chosen = 0;
    for (int n : {1, 2, 4, 8, 16}) {
        const int strip = (rows + n - 1) / n;
        const int min_strip = rows / n;
        int K = want_k > 0 ? want_k : std::min(8, 1 + min_strip / (4 * M));
        if (n == 1) K = want_k > 0 ? want_k : 64;
        const int halo = n == 1 ? M : K * M;
        if (n > 1 && min_strip < halo) continue;
        const size_t smem = cluster_smem_bytes(strip, halo, width, cols);
        if (smem > (size_t)smem_max || !clusters_fit_rule(rule, M, n, smem)) continue;
        ClusterPlan p;
        p.ok = true;
        p.rule = rule;
        p.M = M;
        p.nctas = n;
        p.K = K;
        p.halo = halo;
        p.smem = smem;
        *out = p;
        chosen = n;
        if ((pts + n - 1) / n <= 8LL * kCThreads) break;
    }
    return chosen > 0;
}

cudaError_t launch_cluster_run(const ClusterPlan &p, const Geom &g, const Coef &cf, float adt, float nux, float nuy,
                               float wr, float wc, const float *u0, float *slot0, float *slot1, long long t0,
                               long long nt, double tol, long long *res_steps, double *res_r, cudaStream_t st)
{
    const ClusterArgs a = make_args(p, g);
    RuleArgs ra;
    ra.cf = cf;
    ra.adt = adt;
    ra.nux = nux;
    ra.nuy = nuy;
    ra.wr = wr;
    ra.wc = wc;
    switch (p.rule) {
    case kRuleDiffusion:
        return launch_m<kRuleDiffusion>(p.M, p, a, ra, u0, slot0, slot1, t0, nt, tol, res_steps, res_r, st);
    case kRuleUpwind:
        return launch_m<kRuleUpwind>(p.M, p, a, ra, u0, slot0, slot1, t0, nt, tol, res_steps, res_r, st);
    case kRuleJacobi:
        return launch_m<kRuleJacobi>(p.M, p, a, ra, u0, slot0, slot1, t0, nt, tol, res_steps, res_r, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fdgb
