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
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

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

// Shared memory of the tiled kernel: the u^n ring, the aux ring, the
// mbarriers and the abort flag; then the damping-flag bits of every d0 plane,
// room for src_cap injected corners of the tile and their per-plane starts.
__host__ __device__ inline size_t tma_smem_core(int M, int P, int rows_max)
{
    const int NU = M + 1 + P, NA = P + 1;
    const int box_h = rows_max + 2 * M;
    return sizeof(float) * ((size_t)NU * ring_plane_floats(box_h) + (size_t)NA * 3 * rows_max * kTileW) +
           sizeof(unsigned long long) * (NU + NA) + 16;
}

__host__ __device__ inline size_t tma_smem_bytes(int M, int P, int rows_max, int n0, int src_cap)
{
    return tma_smem_core(M, P, rows_max) + sizeof(unsigned) * (size_t)((n0 + 31) / 32) +
           sizeof(SrcEntry) * (size_t)src_cap + sizeof(int) * (size_t)(n0 + 1);
}

template <int M, int P>
__global__ void __launch_bounds__(16 * kMaxRows, 1)
    acoustic_tma_kernel(const __grid_constant__ CUtensorMap map_u, const __grid_constant__ CUtensorMap map_um,
                        const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_d,
                        float *__restrict__ out, const TileArgs a, const Coef cf, int *status,
                        const unsigned char *__restrict__ dflags, const SrcEntry *__restrict__ src_tab,
                        const int *__restrict__ src_off, const float *__restrict__ src_row, const int src_cap)
{
    constexpr int NU = M + 1 + P;     // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;         // aux planes (u^{n-1}, c, d)
    constexpr int HV = (M + 3) / 4;   // float4 groups on each side of a thread's 4 points
    constexpr int NR = 4 * (2 * HV + 1);
    constexpr int Q = 2 * M + 1;      // d0 queue length; the plane loop is unrolled by Q

    // an earlier launch of this operator gave up on a wait: do nothing until
    // the host has read and cleared the status word
    if (*reinterpret_cast<volatile int *>(status) != 0) return;

    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int box_h = a.box_h;
    const int plane_u = ring_plane_floats(box_h);
    const int plane_a = a.rows_max * kTileW;
    float *ring = reinterpret_cast<float *>(smem_raw);
    float *aux = ring + NU * plane_u;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(aux + NA * 3 * plane_a);
    volatile int *s_abort = reinterpret_cast<volatile int *>(bars + NU + NA);
    unsigned *s_flags = reinterpret_cast<unsigned *>(bars + NU + NA) + 4;
    const int nwords = (a.n0 + 31) / 32;
    SrcEntry *s_src = reinterpret_cast<SrcEntry *>(s_flags + nwords);
    int *s_sstart = reinterpret_cast<int *>(s_src + src_cap);  // plane z's corners: [s_sstart[z], s_sstart[z+1])

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

    // this tile's damping flags (one bit per d0 plane) and injected corners,
    // staged in shared memory so that the plane loop never waits on them
    for (int w = tid; w < nwords; w += blockDim.x) {
        unsigned bits = 0;
        const unsigned char *f = dflags + (long long)blockIdx.x * a.n0 + 32 * w;
        const int nb = min(32, a.n0 - 32 * w);
        for (int b = 0; b < nb; b++) bits |= (f[b] ? 1u : 0u) << b;
        s_flags[w] = bits;
    }
    int nsrc = 0;
    if (src_row) {
        const int s0 = src_off[blockIdx.x];
        nsrc = src_off[blockIdx.x + 1] - s0;
        for (int q = tid; q < nsrc * 5; q += blockDim.x)
            reinterpret_cast<int *>(s_src)[q] = reinterpret_cast<const int *>(src_tab + s0)[q];
    }
    __syncthreads();
    if (nsrc > 0)
        for (int z = tid; z <= a.n0; z += blockDim.x) {
            int lo = 0, hi = nsrc;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_src[mid].z < z) lo = mid + 1; else hi = mid;
            }
            s_sstart[z] = lo;
        }

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
    const uint32_t bytes_box = (uint32_t)(plane_a * sizeof(float));
    auto d_nonzero = [&](int z) -> bool { return (s_flags[z >> 5] >> (z & 31)) & 1u; };

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
            const bool need_d = d_nonzero(ja);
            mbar_expect_tx(ba, (need_d ? 3u : 2u) * bytes_box);
            tma_load_3d(smem_addr(dst), &map_um, col0, row0, ja, ba);
            tma_load_3d(smem_addr(dst + plane_a), &map_c, col0, row0, ja, ba);
            if (need_d) tma_load_3d(smem_addr(dst + 2 * plane_a), &map_d, col0, row0, ja, ba);
        }
    };

    if (tid == 0)
        for (int j = 0; j < P && j < J; j++) issue(j);

    // d0 queue: q[i % Q] holds the thread's 4 centre values of the plane
    // loaded at iteration i; with the loop unrolled by Q every index below is
    // a compile-time constant, so the queue never moves between registers
    float4 q[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);

    int j = 0;
    bool ok = true, stop = false;
    for (int j0 = 0; j0 < J && !stop; j0 += Q) {
#pragma unroll
        for (int jj = 0; jj < Q; jj++) {
            j = j0 + jj;
            if (j >= J) break;
            if (tid == 0 && j + P < J) issue(j + P);
            ok = mbar_wait_bounded(smem_addr(&bars[j % NU]), (uint32_t)((j / NU) & 1)) && ok;
            q[jj] = *reinterpret_cast<const float4 *>(ring + (j % NU) * plane_u + (r + M) * kBoxW + kSideHalo +
                                                      4 * qc);
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
                    const float4 d4 = d_nonzero(ja) ? *reinterpret_cast<const float4 *>(pa + 2 * plane_a)
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
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
                            // planes ja -/+ k were loaded at iterations j - M -/+ k
                            const float4 lo = q[(jj - M - k + 2 * Q) % Q];
                            const float4 hi = q[(jj - M + k + Q) % Q];
                            const float s2 = row[4 * HV + i - k] + row[4 * HV + i + k];
                            const float s1 = (&cm[k].x)[i] + (&cp[k].x)[i];
                            const float s0 = (&lo.x)[i] + (&hi.x)[i];
                            lap = fmaf(cf.ax[2][k], s2, lap);
                            lap = fmaf(cf.ax[1][k], s1, lap);
                            lap = fmaf(cf.ax[0][k], s0, lap);
                        }
                        res[i] = 2.0f * u - umv[i] + cv[i] * lap - dv[i] * (u - umv[i]);
                    }
                    if (nsrc > 0) {
                        // source injection at the corners this thread owns on plane ja
                        float inj0 = 0.f, inj1 = 0.f, inj2 = 0.f, inj3 = 0.f;
                        const int s_end = s_sstart[ja + 1];
                        for (int k = s_sstart[ja]; k < s_end; k++) {
                            const SrcEntry e = s_src[k];
                            if (e.r == r && (e.x >> 2) == qc) {
                                const float sv = e.w * src_row[e.p];
                                const int i = e.x & 3;
                                inj0 += (i == 0) ? sv : 0.f;
                                inj1 += (i == 1) ? sv : 0.f;
                                inj2 += (i == 2) ? sv : 0.f;
                                inj3 += (i == 3) ? sv : 0.f;
                            }
                        }
                        res[0] = fmaf(inj0, cv[0], res[0]);
                        res[1] = fmaf(inj1, cv[1], res[1]);
                        res[2] = fmaf(inj2, cv[2], res[2]);
                        res[3] = fmaf(inj3, cv[3], res[3]);
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
            if (*s_abort) {
                stop = true;
                break;
            }
        }
    }

    if (stop) {
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

// One CTA per (tile, plane block): flags[tile][z] = any d != 0 on the tile's
// rows x 64 columns of plane z; counts the non-zero points.
__global__ void damping_flags_kernel(const TileArgs a, const float *__restrict__ d, unsigned char *flags,
                                     unsigned long long *nz_count)
{
    const int tile = blockIdx.x;
    const int strip = tile / a.k2;
    const int tile2 = tile - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = tile2 * kTileW;
    const int cols = min(kTileW, a.n2 - col0);
    unsigned long long local = 0;
    for (int z = blockIdx.y; z < a.n0; z += gridDim.y) {
        int any = 0;
        for (int q = threadIdx.x; q < rows * cols; q += blockDim.x) {
            const int r = q / cols;
            const int c = q - r * cols;
            const float v = d[(long long)z * a.s0 + (long long)(row0 + r) * a.s1 + col0 + c];
            if (v != 0.0f) {
                any = 1;
                local++;
            }
        }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) flags[(long long)tile * a.n0 + z] = (unsigned char)any;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(nz_count, local);
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

// prefetch depth: planes in flight per CTA; the kernel is latency-bound
// below ~4 (one CTA per SM keeps P x (haloed u^n + u^{n-1}, c, d tiles) in
// flight), so the planner takes the deepest that fits
constexpr int kMinStages = 2;
constexpr int kMaxStages = 4;
constexpr size_t kSparseReserve = 16 * 1024;  // shared memory kept for fused point lists

template <int M>
cudaError_t configure_kernel(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(acoustic_tma_kernel<M, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(acoustic_tma_kernel<M, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(acoustic_tma_kernel<M, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

}  // namespace

fd_status tma_plan_build(TmaPlan &plan, int kind, int space_order, const Geom &g, float *const slot[2], float *c,
                         float *d)
{
    const int want_rows = plan.force_rows, want_stages = plan.force_stages;
    plan.ready = false;
    if (kind != FD_ACOUSTIC_LEAPFROG || g.ndim != 3) return FD_OK;
    const int M = space_order / 2;
    if (g.n[0] > (1 << 30) || g.n[1] > (1 << 30) || g.n[2] > (1 << 30)) return FD_OK;
    int dev = 0, sms = 0, smem_max = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(FD_ERR_CUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (sms <= 0 || smem_max <= 0 || smem_sm <= 0) return set_error(FD_ERR_CUDA, "device attributes unavailable");

    TileArgs a{};
    a.n0 = (int)g.n[0];
    a.n1 = (int)g.n[1];
    a.n2 = (int)g.n[2];
    a.s0 = g.s0;
    a.s1 = g.s1;
    a.k2 = (a.n2 + kTileW - 1) / kTileW;
    // CTAs resident per SM for a tile height (shared memory and threads)
    auto occupancy = [&](int rows, int P) {
        const size_t per = tma_smem_bytes(M, P, rows, a.n0, 0) + 1024;
        int occ = (int)((size_t)smem_sm / per);
        occ = std::min(occ, 2048 / (16 * rows));
        return std::max(occ, 0);
    };
    // Choose the strip count k1 (tile height rows = ceil(n1/k1)): minimise the
    // work of the busiest SM, ceil(ctas / SMs) tiles of rows + M/2 row-planes
    // (halo rows cost TMA traffic, served mostly from L2), with every tile of
    // one wave resident at once; ties go to taller tiles.
    int best_k1 = -1;
    double best_cost = 0;
    if (want_rows > 0) {
        const int k1 = (a.n1 + want_rows - 1) / want_rows;
        if (want_rows > kMaxRows || occupancy((a.n1 + k1 - 1) / k1, kMinStages) < 1)
            return set_error(FD_ERR_UNSUPPORTED, "tiling: %d rows per tile do not fit", want_rows);
        best_k1 = k1;
    } else {
        for (int k1 = (a.n1 + kMaxRows - 1) / kMaxRows; k1 <= a.n1; k1++) {
            const int rows_max = (a.n1 + k1 - 1) / k1;
            const int occ = occupancy(rows_max, kMinStages);
            if (occ < 1) continue;
            const long long ctas = (long long)k1 * a.k2;
            const long long per_sm = (ctas + sms - 1) / sms;
            const long long waves = (per_sm + occ - 1) / occ;
            const double cost = (double)waves * occ * (rows_max + 0.5 * M) * (per_sm > occ ? 1.0 : (double)per_sm / occ);
            if (best_k1 < 0 || cost < best_cost - 1e-9) {
                best_k1 = k1;
                best_cost = cost;
            }
            if (ctas > 8LL * sms) break;
        }
    }
    if (best_k1 < 0) return FD_OK;  // tiles do not fit: plain kernels
    a.k1 = best_k1;
    a.rows_max = (a.n1 + a.k1 - 1) / a.k1;
    a.box_h = a.rows_max + 2 * M;

    // deepest prefetch that keeps the occupancy of the minimum depth
    const int occ2 = occupancy(a.rows_max, kMinStages);
    int P = kMinStages;
    for (int p = kMaxStages; p > kMinStages; p--)
        if (occupancy(a.rows_max, p) >= occ2 &&
            tma_smem_bytes(M, p, a.rows_max, a.n0, 0) + kSparseReserve <= (size_t)smem_max) {
            P = p;
            break;
        }
    if (want_stages > 0) {
        if (want_stages < kMinStages || want_stages > kMaxStages ||
            tma_smem_bytes(M, want_stages, a.rows_max, a.n0, 0) > (size_t)smem_max)
            return set_error(FD_ERR_UNSUPPORTED, "tiling: %d stages do not fit", want_stages);
        P = want_stages;
    }

    plan.kind = kind;
    plan.M = M;
    plan.stages = P;
    plan.args = a;
    plan.threads = 16 * a.rows_max;
    plan.smem = tma_smem_bytes(M, P, a.rows_max, a.n0, 0);
    plan.smem_max = (size_t)smem_max;
    plan.src_cap = 0;
    plan.slot[0] = slot[0];
    plan.slot[1] = slot[1];
    plan.d = d;
    if (!plan.dflags) {
        // (k1*k2) x n0 bytes plus the non-zero counter
        size_t bytes = (size_t)a.k1 * a.k2 * a.n0 + 16;
        if (cudaMalloc((void **)&plan.dflags, bytes) != cudaSuccess)
            return set_error(FD_ERR_NOMEM, "tiled plan: damping flags");
        plan.nz_count = (unsigned long long *)(plan.dflags + ((size_t)a.k1 * a.k2 * a.n0 + 7) / 8 * 8);
        if (cudaMemset(plan.dflags, 1, (size_t)a.k1 * a.k2 * a.n0) != cudaSuccess)
            return set_error(FD_ERR_CUDA, "tiled plan: damping flags");
    }
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

void tma_plan_release(TmaPlan &plan, cudaStream_t st)
{
    plan.ready = false;
    if (plan.dflags || plan.fused_mem) cudaStreamSynchronize(st);
    if (plan.dflags) cudaFree(plan.dflags);
    if (plan.fused_mem) cudaFree(plan.fused_mem);
    plan.dflags = nullptr;
    plan.nz_count = nullptr;
    plan.fused_mem = nullptr;
    plan.fused = SparseFused();
    plan.has_src = false;
}

fd_status tma_sparse_build(TmaPlan &plan, const SparseHostView *src, cudaStream_t st)
{
    if (plan.fused_mem) {
        cudaStreamSynchronize(st);
        cudaFree(plan.fused_mem);
        plan.fused_mem = nullptr;
    }
    plan.has_src = false;
    plan.fused = SparseFused();
    plan.src_cap = 0;
    if (!plan.ready) return FD_OK;
    const TileArgs &a = plan.args;
    const int M = plan.M;
    const int tiles = a.k1 * a.k2;
    plan.smem = tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, 0);
    if (!src || src->npoint <= 0) return FD_OK;
    // tile owning grid row i1 and column i2, and that tile's first row/column
    auto owner = [&](int64_t i1, int64_t i2, int &tile, int &row0, int &col0) {
        int strip = (int)(i1 * a.k1 / a.n1);
        while (strip > 0 && (int64_t)strip * a.n1 / a.k1 > i1) strip--;
        while (strip + 1 < a.k1 && (int64_t)(strip + 1) * a.n1 / a.k1 <= i1) strip++;
        const int t2 = (int)(i2 / kTileW);
        row0 = (int)((int64_t)strip * a.n1 / a.k1);
        col0 = t2 * kTileW;
        tile = strip * a.k2 + t2;
    };
    std::vector<std::vector<SrcEntry>> per(tiles);
    for (int p = 0; p < src->npoint; p++) {
        const int64_t lin = src->base[p];
        const int64_t i0 = lin / a.s0;
        const int64_t rem = lin - i0 * a.s0;
        const int64_t i1 = rem / a.s1;
        const int64_t i2 = rem - i1 * a.s1;
        for (int k = 0; k < 8; k++) {
            const float w = src->weight[(size_t)p * 8 + k];
            if (w == 0.0f) continue;
            const int64_t z = i0 + (k & 1), y = i1 + ((k >> 1) & 1), x = i2 + ((k >> 2) & 1);
            int tile, row0, col0;
            owner(y, x, tile, row0, col0);
            SrcEntry e;
            e.z = (int)z;
            e.r = (int)(y - row0);
            e.x = (int)(x - col0);
            e.p = p;
            e.w = w;
            per[tile].push_back(e);
        }
    }
    std::vector<int> off(tiles + 1, 0);
    std::vector<SrcEntry> all;
    size_t max_s = 0;
    for (int t = 0; t < tiles; t++) {
        std::stable_sort(per[t].begin(), per[t].end(), [](const SrcEntry &x, const SrcEntry &y) { return x.z < y.z; });
        off[t] = (int)all.size();
        all.insert(all.end(), per[t].begin(), per[t].end());
        max_s = std::max(max_s, per[t].size());
    }
    off[tiles] = (int)all.size();
    // the tile's corners are staged in shared memory: lower the prefetch depth
    // if that is what it takes, else leave injection to its own kernel
    while (plan.stages > kMinStages &&
           tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, (int)max_s) > plan.smem_max)
        plan.stages--;
    if (tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, (int)max_s) > plan.smem_max) {
        plan.smem = tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, 0);
        return FD_OK;
    }
    const size_t b_src = (sizeof(SrcEntry) * all.size() + 15) / 16 * 16;
    const size_t b_off = sizeof(int) * (tiles + 1);
    unsigned char *mem = nullptr;
    if (cudaMalloc((void **)&mem, b_src + b_off + 16) != cudaSuccess) return set_error(FD_ERR_NOMEM, "fused sources");
    plan.fused_mem = mem;
    cudaError_t e = cudaMemcpyAsync(mem, all.data(), sizeof(SrcEntry) * all.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mem + b_src, off.data(), b_off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fused sources: %s", cudaGetErrorString(e));
    plan.fused.src = (const SrcEntry *)mem;
    plan.fused.src_off = (const int *)(mem + b_src);
    plan.has_src = true;
    plan.src_cap = (int)max_s;
    plan.smem = tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, plan.src_cap);
    return FD_OK;
}

void tma_plan_tiling(const TmaPlan &plan, int *rows, int *stages, int *ctas)
{
    *rows = plan.ready ? plan.args.rows_max : 0;
    *stages = plan.ready ? plan.stages : 0;
    *ctas = plan.ready ? plan.args.k1 * plan.args.k2 : 0;
}

cudaError_t launch_damping_flags(const TmaPlan &plan, cudaStream_t st)
{
    const TileArgs &a = plan.args;
    cudaError_t e = cudaMemsetAsync(plan.nz_count, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int tiles = a.k1 * a.k2;
    int zblocks = (152 * 8 + tiles - 1) / tiles;
    if (zblocks > a.n0) zblocks = a.n0;
    damping_flags_kernel<<<dim3((unsigned)tiles, (unsigned)zblocks), 256, 0, st>>>(a, plan.d, plan.dflags,
                                                                                   plan.nz_count);
    return cudaGetLastError();
}

static cudaError_t launch_maps(const TmaPlan &plan, int M, const Coef &cf, const CUtensorMap &map_cur,
                               const CUtensorMap &map_prev, float *out, int *status, const float *src_row,
                               cudaStream_t st)
{
    dim3 grid((unsigned)(plan.args.k1 * plan.args.k2));
    dim3 block((unsigned)plan.threads);
    const float *srow = plan.has_src ? src_row : nullptr;
    const int key = M * 8 + plan.stages;
    switch (key) {
#define CASE(MM, PP)                                                                                      \
    case MM * 8 + PP:                                                                                     \
        acoustic_tma_kernel<MM, PP><<<grid, block, plan.smem, st>>>(                                      \
            map_cur, map_prev, plan.c_tile, plan.d_tile, out, plan.args, cf, status, plan.dflags,         \
            plan.fused.src, plan.fused.src_off, srow, plan.src_cap);                                      \
        break;
#define CASES(MM) CASE(MM, 2) CASE(MM, 3) CASE(MM, 4)
        CASES(1) CASES(2) CASES(3) CASES(4) CASES(5) CASES(6) CASES(7) CASES(8)
#undef CASES
#undef CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_acoustic_tma(const TmaPlan &plan, int M, const Geom &g, const Coef &cf, int cur, int *status,
                                const float *src_row, cudaStream_t st)
{
    (void)g;
    const int prev = cur ^ 1;
    return launch_maps(plan, M, cf, plan.u_halo[cur], plan.u_tile[prev], plan.slot[prev], status, src_row, st);
}

static const CUtensorMap *cached_map(TmaPlan &plan, const float *ptr, bool halo)
{
    for (auto &e : plan.cache)
        if (e.ptr == ptr && e.halo == halo) return &e.map;
    TmaPlan::CachedMap e;
    e.ptr = ptr;
    e.halo = halo;
    if (encode_3d(&e.map, const_cast<float *>(ptr), plan.args, halo ? kBoxW : kTileW,
                  halo ? plan.args.box_h : plan.args.rows_max) != FD_OK)
        return nullptr;
    if (plan.cache.size() >= 512) plan.cache.erase(plan.cache.begin());
    plan.cache.push_back(e);
    return &plan.cache.back().map;
}

cudaError_t launch_acoustic_tma_buffers(TmaPlan &plan, int M, const Coef &cf, const float *u_cur, const float *u_prev,
                                        float *u_next, int *status, const float *src_row, cudaStream_t st)
{
    const CUtensorMap *mc = cached_map(plan, u_cur, true);
    if (!mc) return cudaErrorInvalidValue;
    const CUtensorMap map_cur = *mc;  // copy: the next lookup may move the cache
    const CUtensorMap *mp = cached_map(plan, u_prev, false);
    if (!mp) return cudaErrorInvalidValue;
    return launch_maps(plan, M, cf, map_cur, *mp, u_next, status, src_row, st);
}

}  // namespace fdgb
