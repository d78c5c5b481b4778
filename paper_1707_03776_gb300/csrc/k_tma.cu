// Tiled acoustic step for 3D grids: 2.5D blocking with TMA-staged tiles.
//
// Each CTA owns one tile column -- rows [row0, row0+rows) of d1 and 64
// columns of d2 -- and sweeps every d0 plane of it.  Per plane:
//   * one TMA box brings the haloed u^n tile (64+16 columns, rows+2M rows)
//     into a ring of shared-memory planes; the zero halo around the grid is
//     the TMA out-of-bounds fill, so no halo is stored in HBM;
//   * three TMA boxes bring u^{n-1}, c = dt^2/m and d = dt*eta/m of the plane
//     being finished into a second ring;
//   * every thread owns 4 consecutive d2 points of one row, keeps the 2M+1
//     centre values along d0 in a register queue, reads the d1/d2 neighbours
//     of the plane M behind the newest from shared memory, and writes u^{n+1}
//     over u^{n-1} with 128-bit stores.
// One elected thread issues the copies P planes ahead, on mbarriers with
// transaction counts; every wait is bounded by the global timer and, when it
// gives up, the CTA records FD_ERR_TIMEOUT in the operator's status word and
// leaves after draining its own copies.
//
// The grid has one CTA per tile, and the planner sizes the tiles so that the
// tile count matches the SM count (152 on GB300): all CTAs sweep d0 together,
// so the halo rows a CTA loads were just loaded by its neighbour and are
// served from L2.
#include <cstdio>
#include <cstring>

#include "fd_internal_host.h"
#include "fd_tma.h"

namespace fdgb {

namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of a barrier, giving up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(map)) : "memory");
}

__host__ __device__ constexpr int round_up32(int x) { return (x + 31) / 32 * 32; }

// floats of one ring plane (rounded so every plane starts 128-byte aligned)
__host__ __device__ inline int ring_plane_floats(int box_h) { return round_up32(box_h * kBoxW); }

__host__ __device__ inline size_t tma_smem_bytes(int M, int P, int rows_max)
{
    const int NU = M + 1 + P, NA = P + 1;
    const int box_h = rows_max + 2 * M;
    return sizeof(float) * ((size_t)NU * ring_plane_floats(box_h) + (size_t)NA * 3 * rows_max * kTileW) +
           sizeof(unsigned long long) * (NU + NA) + 16;
}

template <int M, int P>
__global__ void __launch_bounds__(16 * kMaxRows, 1)
    acoustic_tma_kernel(const __grid_constant__ CUtensorMap map_u, const __grid_constant__ CUtensorMap map_um,
                        const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_d,
                        float *__restrict__ out, const TileArgs a, const Coef cf, int *status)
{
    constexpr int NU = M + 1 + P;     // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;         // aux planes (u^{n-1}, c, d)
    constexpr int HV = (M + 3) / 4;   // float4 groups on each side of a thread's 4 points
    constexpr int NR = 4 * (2 * HV + 1);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int box_h = a.box_h;
    const int plane_u = ring_plane_floats(box_h);
    const int plane_a = a.rows_max * kTileW;
    float *ring = reinterpret_cast<float *>(smem_raw);
    float *aux = ring + NU * plane_u;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(aux + NA * 3 * plane_a);
    volatile int *s_abort = reinterpret_cast<volatile int *>(bars + NU + NA);

    // an earlier launch of this operator gave up on a wait: do nothing until
    // the host has read and cleared the status word
    if (*reinterpret_cast<volatile int *>(status) != 0) return;

    const int tid = threadIdx.x;
    const int strip = blockIdx.x / a.k2;
    const int tile2 = blockIdx.x - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = tile2 * kTileW;
    const int r = tid >> 4;
    const int qc = tid & 15;
    const bool active = r < rows && col0 + 4 * qc < a.n2;
    const int J = a.n0 + 2 * M;

    if (tid == 0) {
        prefetch_map(&map_u);
        prefetch_map(&map_um);
        prefetch_map(&map_c);
        prefetch_map(&map_d);
        for (int i = 0; i < NU + NA; i++) mbar_init(smem_addr(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s_abort = 0;
    }
    __syncthreads();

    const uint32_t bytes_u = (uint32_t)(kBoxW * box_h * sizeof(float));
    const uint32_t bytes_a = (uint32_t)(3 * plane_a * sizeof(float));

    // iteration j: u^n plane j-M into ring slot j % NU; for j >= 2M the aux of
    // output plane j-2M into aux slot (j-2M) % NA
    auto issue = [&](int j) {
        const int su = j % NU;
        const uint32_t bu = smem_addr(&bars[su]);
        mbar_expect_tx(bu, bytes_u);
        tma_load_3d(smem_addr(ring + su * plane_u), &map_u, col0 - kSideHalo, row0 - M, j - M, bu);
        if (j >= 2 * M) {
            const int ja = j - 2 * M;
            const int sa = ja % NA;
            const uint32_t ba = smem_addr(&bars[NU + sa]);
            float *dst = aux + sa * 3 * plane_a;
            mbar_expect_tx(ba, bytes_a);
            tma_load_3d(smem_addr(dst), &map_um, col0, row0, ja, ba);
            tma_load_3d(smem_addr(dst + plane_a), &map_c, col0, row0, ja, ba);
            tma_load_3d(smem_addr(dst + 2 * plane_a), &map_d, col0, row0, ja, ba);
        }
    };

    if (tid == 0)
        for (int j = 0; j < P && j < J; j++) issue(j);

    float4 q[2 * M + 1];
#pragma unroll
    for (int k = 0; k <= 2 * M; k++) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);

    int j = 0;
    bool ok = true;
    for (; j < J; j++) {
        if (tid == 0 && j + P < J) issue(j + P);
        ok = mbar_wait_bounded(smem_addr(&bars[j % NU]), (uint32_t)((j / NU) & 1)) && ok;

        // push the centre values of plane j-M onto the d0 queue
#pragma unroll
        for (int k = 0; k < 2 * M; k++) q[k] = q[k + 1];
        const float *pnew = ring + (j % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc;
        q[2 * M] = *reinterpret_cast<const float4 *>(pnew);

        if (j >= 2 * M) {
            const int ja = j - 2 * M;  // output plane
            ok = mbar_wait_bounded(smem_addr(&bars[NU + ja % NA]), (uint32_t)((ja / NA) & 1)) && ok;
            if (ok && active) {
                const float *pc = ring + ((j - M) % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc;
                float row[NR];
#pragma unroll
                for (int v = 0; v < 2 * HV + 1; v++) {
                    float4 t = *reinterpret_cast<const float4 *>(pc + 4 * (v - HV));
                    row[4 * v + 0] = t.x;
                    row[4 * v + 1] = t.y;
                    row[4 * v + 2] = t.z;
                    row[4 * v + 3] = t.w;
                }
                float4 cm[M + 1], cp[M + 1];
#pragma unroll
                for (int k = 1; k <= M; k++) {
                    cm[k] = *reinterpret_cast<const float4 *>(pc - k * kBoxW);
                    cp[k] = *reinterpret_cast<const float4 *>(pc + k * kBoxW);
                }
                const float *pa = aux + (ja % NA) * 3 * plane_a + r * kTileW + 4 * qc;
                const float4 um4 = *reinterpret_cast<const float4 *>(pa);
                const float4 c4 = *reinterpret_cast<const float4 *>(pa + plane_a);
                const float4 d4 = *reinterpret_cast<const float4 *>(pa + 2 * plane_a);
                const float umv[4] = {um4.x, um4.y, um4.z, um4.w};
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
                float res[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float u = row[4 * HV + i];
                    float lap = cf.centre * u;
#pragma unroll
                    for (int k = 1; k <= M; k++) {
                        const float s2 = row[4 * HV + i - k] + row[4 * HV + i + k];
                        const float s1 = (&cm[k].x)[i] + (&cp[k].x)[i];
                        const float s0 = (&q[M - k].x)[i] + (&q[M + k].x)[i];
                        lap = fmaf(cf.ax[2][k], s2, lap);
                        lap = fmaf(cf.ax[1][k], s1, lap);
                        lap = fmaf(cf.ax[0][k], s0, lap);
                    }
                    res[i] = 2.0f * u - umv[i] + cv[i] * lap - dv[i] * (u - umv[i]);
                }
                float *o = out + (long long)ja * a.s0 + (long long)(row0 + r) * a.s1 + col0 + 4 * qc;
                if (col0 + 4 * qc + 3 < a.n2) {
                    *reinterpret_cast<float4 *>(o) = make_float4(res[0], res[1], res[2], res[3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++)
                        if (col0 + 4 * qc + i < a.n2) o[i] = res[i];
                }
            }
        }
        if (!ok) *s_abort = 1;
        __syncthreads();
        if (*s_abort) break;
    }

    if (j < J) {
        // a wait gave up: record it, then drain this CTA's copies still in
        // flight (issued up to min(j+P, J-1)) before leaving
        if (tid == 0) {
            atomicExch(status, (int)FD_ERR_TIMEOUT);
            const int last = (j + P < J) ? j + P : J - 1;
            for (int i = j; i <= last; i++) {
                if (!mbar_wait_bounded(smem_addr(&bars[i % NU]), (uint32_t)((i / NU) & 1))) break;
                if (i >= 2 * M) {
                    const int ia = i - 2 * M;
                    if (!mbar_wait_bounded(smem_addr(&bars[NU + ia % NA]), (uint32_t)((ia / NA) & 1))) break;
                }
            }
        }
        __syncthreads();
    }
}

// ---- host side ---------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

fd_status encode_3d(CUtensorMap *map, float *base, const TileArgs &a, int box_w, int box_h)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {(cuuint64_t)a.n2, (cuuint64_t)a.n1, (cuuint64_t)a.n0};
    cuuint64_t strides[2] = {(cuuint64_t)a.s1 * sizeof(float), (cuuint64_t)a.s0 * sizeof(float)};
    cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FD_OK;
}

constexpr int kStages = 2;

template <int M>
cudaError_t configure_kernel(size_t smem)
{
    return cudaFuncSetAttribute(acoustic_tma_kernel<M, kStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

}  // namespace

fd_status tma_plan_build(TmaPlan &plan, int kind, int space_order, const Geom &g, float *const slot[2], float *c,
                         float *d)
{
    plan.ready = false;
    if (kind != FD_ACOUSTIC_LEAPFROG || g.ndim != 3) return FD_OK;
    const int M = space_order / 2;
    if (g.n[0] > (1 << 30) || g.n[1] > (1 << 30) || g.n[2] > (1 << 30)) return FD_OK;
    int dev = 0, sms = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(FD_ERR_CUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sms <= 0 || smem_max <= 0) return set_error(FD_ERR_CUDA, "device attributes unavailable");

    TileArgs a{};
    a.n0 = (int)g.n[0];
    a.n1 = (int)g.n[1];
    a.n2 = (int)g.n[2];
    a.s0 = g.s0;
    a.s1 = g.s1;
    a.k2 = (a.n2 + kTileW - 1) / kTileW;
    // Choose the number of d1 strips: minimise (waves x per-CTA rows), one CTA per SM.
    int best_k1 = -1;
    long long best_cost = 0;
    for (int k1 = (a.n1 + kMaxRows - 1) / kMaxRows; k1 <= a.n1; k1++) {
        const int rows_max = (a.n1 + k1 - 1) / k1;
        if (tma_smem_bytes(M, kStages, rows_max) > (size_t)smem_max) continue;
        const long long ctas = (long long)k1 * a.k2;
        const long long waves = (ctas + sms - 1) / sms;
        const long long cost = waves * rows_max;
        if (best_k1 < 0 || cost < best_cost) {
            best_k1 = k1;
            best_cost = cost;
        }
        if (ctas > 4LL * sms) break;
    }
    if (best_k1 < 0) return FD_OK;  // tiles do not fit: plain kernels
    a.k1 = best_k1;
    a.rows_max = (a.n1 + a.k1 - 1) / a.k1;
    a.box_h = a.rows_max + 2 * M;

    plan.kind = kind;
    plan.M = M;
    plan.stages = kStages;
    plan.args = a;
    plan.threads = 16 * a.rows_max;
    plan.smem = tma_smem_bytes(M, kStages, a.rows_max);
    plan.slot[0] = slot[0];
    plan.slot[1] = slot[1];
    for (int s = 0; s < 2; s++) {
        fd_status st = encode_3d(&plan.u_halo[s], slot[s], a, kBoxW, a.box_h);
        if (st != FD_OK) return st;
        st = encode_3d(&plan.u_tile[s], slot[s], a, kTileW, a.rows_max);
        if (st != FD_OK) return st;
    }
    fd_status st = encode_3d(&plan.c_tile, c, a, kTileW, a.rows_max);
    if (st != FD_OK) return st;
    st = encode_3d(&plan.d_tile, d, a, kTileW, a.rows_max);
    if (st != FD_OK) return st;
    // the attribute is the per-launch ceiling, not the request: set it to the
    // device limit so operators of different tile heights can coexist
    cudaError_t e = cudaErrorInvalidValue;
    switch (M) {
#define CASE(MM) \
    case MM: e = configure_kernel<MM>((size_t)smem_max); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    if (e != cudaSuccess)
        return set_error(FD_ERR_CUDA, "tiled kernel configuration: %s", cudaGetErrorString(e));
    plan.ready = true;
    return FD_OK;
}

void tma_plan_release(TmaPlan &plan) { plan.ready = false; }

cudaError_t launch_acoustic_tma(const TmaPlan &plan, int M, const Geom &g, const Coef &cf, int cur, int *status,
                                cudaStream_t st)
{
    (void)g;
    const int prev = cur ^ 1;
    dim3 grid((unsigned)(plan.args.k1 * plan.args.k2));
    dim3 block((unsigned)plan.threads);
    float *out = plan.slot[prev];
    switch (M) {
#define CASE(MM)                                                                                          \
    case MM:                                                                                              \
        acoustic_tma_kernel<MM, kStages><<<grid, block, plan.smem, st>>>(                                 \
            plan.u_halo[cur], plan.u_tile[prev], plan.c_tile, plan.d_tile, out, plan.args, cf, status);   \
        break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace fdgb
