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
// The grid has one CTA per tile and d0 chunk, and the planner sizes the
// tiles (and, for grids too small to fill the GPU with columns, splits d0
// into chunks) so that the CTA count matches the resident slots of the 152
// SMs: all CTAs sweep together, so the halo rows a CTA loads were just loaded
// by its neighbour and are served from L2.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fd_internal_host.h"
#include "fd_tma.h"
#include "k_sweep.cuh"

namespace fdgb {

namespace {

using namespace tile_dev;

template <int M, int P, bool IMG>
__global__ void __launch_bounds__(16 * kMaxRowsTiled + 32, 1)
    acoustic_tma_kernel(const __grid_constant__ CUtensorMap map_u, const __grid_constant__ CUtensorMap map_um,
                        const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_d,
                        float *__restrict__ out, const TileArgs a, const Coef cf, int *status,
                        const SrcEntry *__restrict__ src_tab, const int *__restrict__ src_off,
                        const float *__restrict__ src_row, const int src_cap, const ImagingArgs img)
{
    // an earlier launch of this operator gave up on a wait: do nothing until
    // the host has read and cleared the status word
    if (*reinterpret_cast<volatile int *>(status) != 0) return;
    if (!smem_fits<M, P>(a.rows_max, src_cap, a.n0, status)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const SweepSmem sm = carve_smem<M, P>(smem_raw, a.rows_max, src_cap);
    if (threadIdx.x == 0) {
        prefetch_map(&map_u);
        prefetch_map(&map_um);
        prefetch_map(&map_c);
        prefetch_map(&map_d);
    }
    init_barriers_ws<M, P>(sm, (blockDim.x >> 5) - 1);
    // CTA = (d0 chunk, tile column); chunks are balanced ranges of planes
    const int ncol = a.k1 * a.k2;
    const int tile = (int)(blockIdx.x % (unsigned)ncol);
    const int chunk = (int)(blockIdx.x / (unsigned)ncol);
    const int z_lo = (int)((long long)chunk * a.n0 / a.kz);
    const int z_hi = (int)((long long)(chunk + 1) * a.n0 / a.kz);
    const int item = tile * a.kz + chunk;  // the CTA's own corner list
    const int s0 = src_row ? src_off[item] : 0;
    const int nsrc = src_row ? src_off[item + 1] - s0 : 0;
    if (nsrc > src_cap) {
        // more corners than the launch staged room for
        if (threadIdx.x == 0) atomicExch(status, (int)FD_ERR_LAYOUT);
        return;
    }
    sweep_column_ws<M, P, IMG>(&map_u, &map_um, &map_c, &map_d, out, a, cf, tile, z_lo, z_hi, src_tab + s0, nsrc,
                               src_row, sm, status, img);
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

// prefetch depth: planes in flight per CTA.  The planner takes the deepest
// up to kPlanStages that keeps the CTAs per SM of the minimum depth (on 512^3
// a fourth plane was never faster than a third, and costs shared memory);
// fd_operator_set_tiling may ask for up to kMaxStages.
constexpr int kMinStages = 2;
constexpr int kPlanStages = 3;
constexpr int kMaxStages = 4;
constexpr size_t kSparseReserve = 16 * 1024;  // shared memory kept for fused point lists

template <int M>
cudaError_t configure_kernel(size_t smem)
{
    cudaError_t e = cudaSuccess;
    auto set = [&](auto kernel) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    };
    set(acoustic_tma_kernel<M, 2, false>);
    set(acoustic_tma_kernel<M, 3, false>);
    set(acoustic_tma_kernel<M, 4, false>);
    set(acoustic_tma_kernel<M, 2, true>);
    set(acoustic_tma_kernel<M, 3, true>);
    set(acoustic_tma_kernel<M, 4, true>);
    return e;
}

}  // namespace

fd_status tma_encode_3d(CUtensorMap *map, float *base, const TileArgs &a, int box_w, int box_h)
{
    return encode_3d(map, base, a, box_w, box_h);
}

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
        occ = std::min(occ, 2048 / tma_threads(rows));
        return std::max(occ, 0);
    };
    // Choose the strip count k1 (tile height rows = ceil(n1/k1)): minimise the
    // work of the busiest SM, ceil(ctas / SMs) tiles of rows + 4M row-planes
    // (the 2M halo rows of a box cost about twice an interior row: TMA
    // traffic served from L2 and the barrier wait for it), with every tile of
    // one wave resident at once.  Two or more CTAs sharing an SM hide each
    // other's per-plane barrier waits, worth a factor 1.5 for M >= 2 (at SO2
    // one CTA of tall tiles per SM measured best; sweeps of tile height and
    // depth at 128^3-512^3, SO 2-16).  Ties go to taller tiles.
    // The d0 chunk count kz multiplies the CTAs only for grids whose columns
    // alone leave SMs idle (up to the resident slots of all SMs); a chunk
    // costs its planes plus the 2M it loads before its first output plane
    // (weighted 0.35: u^n is one of the four streams).  Chunks keep at least
    // 4M planes.
    const int kz_lim = std::max(1, std::min(64, a.n0 / std::max(4 * M, 8)));
    auto kz_cap = [&](int k1, int occ) {
        const long long cols = (long long)k1 * a.k2;
        if (cols >= sms) return 1;
        return (int)std::min<long long>(kz_lim, ((long long)sms * occ + cols - 1) / cols);
    };
    auto cost_of = [&](int k1, int kz, int occ) {
        const int rows_max = (a.n1 + k1 - 1) / k1;
        const long long ctas = (long long)k1 * a.k2 * kz;
        const long long per_sm = (ctas + sms - 1) / sms;
        const long long waves = (per_sm + occ - 1) / occ;
        const double planes = (double)((a.n0 + kz - 1) / kz) + 0.35 * 2 * M;
        const long long resident = per_sm < occ ? per_sm : occ;
        const double overlap = resident >= 2 && M >= 2 ? 1.5 : 1.0;
        return (double)waves * occ * (rows_max + 4.0 * M) * planes * (per_sm > occ ? 1.0 : (double)per_sm / occ) /
               overlap;
    };
    int best_k1 = -1, best_kz = 1;
    double best_cost = 0;
    if (want_rows > 0) {
        const int k1 = (a.n1 + want_rows - 1) / want_rows;
        const int occ = occupancy((a.n1 + k1 - 1) / k1, kMinStages);
        if (want_rows > kMaxRowsTiled || occ < 1)
            return set_error(FD_ERR_UNSUPPORTED, "tiling: %d rows per tile do not fit", want_rows);
        best_k1 = k1;
        for (int kz = 1; kz <= kz_cap(k1, occ); kz++) {
            const double cost = cost_of(k1, kz, occ);
            if (kz == 1 || cost < best_cost - 1e-9) {
                best_kz = kz;
                best_cost = cost;
            }
        }
    } else {
        for (int k1 = (a.n1 + kMaxRowsTiled - 1) / kMaxRowsTiled; k1 <= a.n1; k1++) {
            const int rows_max = (a.n1 + k1 - 1) / k1;
            const int occ = occupancy(rows_max, kMinStages);
            if (occ < 1) continue;
            for (int kz = 1; kz <= kz_cap(k1, occ); kz++) {
                const double cost = cost_of(k1, kz, occ);
                if (best_k1 < 0 || cost < best_cost - 1e-9) {
                    best_k1 = k1;
                    best_kz = kz;
                    best_cost = cost;
                }
            }
            if ((long long)k1 * a.k2 > 8LL * sms) break;
        }
    }
    if (best_k1 < 0) return FD_OK;  // tiles do not fit: plain kernels
    a.k1 = best_k1;
    a.kz = best_kz;
    a.stall_plane = plan.stall_plane;
    a.rows_max = (a.n1 + a.k1 - 1) / a.k1;
    a.box_h = a.rows_max + 2 * M;

    // deepest prefetch that still holds, per SM, the CTAs of one wave at the
    // minimum depth (the tiling may place fewer per SM than fit)
    const long long ctas = (long long)a.k1 * a.k2 * a.kz;
    const int occ2 = occupancy(a.rows_max, kMinStages);
    const int need = (int)std::min<long long>(occ2, (ctas + sms - 1) / sms);
    int P = kMinStages;
    for (int p = kPlanStages; p > kMinStages; p--)
        if (occupancy(a.rows_max, p) >= need &&
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
    plan.threads = tma_threads(a.rows_max);
    plan.smem = tma_smem_bytes(M, P, a.rows_max, a.n0, 0);
    plan.smem_max = (size_t)smem_max;
    plan.src_cap = 0;
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

void tma_plan_release(TmaPlan &plan, cudaStream_t st)
{
    plan.ready = false;
    if (plan.fused_mem) {
        cudaStreamSynchronize(st);
        cudaFree(plan.fused_mem);
    }
    plan.fused_mem = nullptr;
    plan.fused = SparseFused();
    plan.has_src = false;
}

void fused_corner_lists(const TileArgs &a, int kz, const SparseHostView *src, std::vector<SrcEntry> &all,
                        std::vector<int> &off, int &max_per_item, int &max_per_column)
{
    const int tiles = a.k1 * a.k2;
    const int items = tiles * kz;
    all.clear();
    off.assign(items + 1, 0);
    max_per_item = 0;
    max_per_column = 0;
    if (!src || src->npoint <= 0) return;
    // the d0 chunk holding plane z: chunk c covers [c n0 / kz, (c + 1) n0 / kz)
    auto chunk_of = [&](int64_t z) {
        int c = (int)(z * kz / a.n0);
        while (c > 0 && (int64_t)c * a.n0 / kz > z) c--;
        while (c + 1 < kz && (int64_t)(c + 1) * a.n0 / kz <= z) c++;
        return c;
    };
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
    std::vector<std::vector<SrcEntry>> per(items);
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
            per[(size_t)tile * kz + chunk_of(z)].push_back(e);
        }
    }
    // item (tile t, chunk c) = t kz + c: a tile's chunks are consecutive, so a
    // whole column's corners are one run as well (the batched kernel sweeps
    // whole columns)
    for (int it = 0; it < items; it++) {
        // by plane, then by the thread owning the corner (row, 4-column
        // group): a thread finds its entries by binary search; stable, so the
        // entries of one point stay in (point, corner) order
        std::stable_sort(per[it].begin(), per[it].end(), [](const SrcEntry &x, const SrcEntry &y) {
            return x.z != y.z ? x.z < y.z : src_owner_key(x) < src_owner_key(y);
        });
        off[it] = (int)all.size();
        all.insert(all.end(), per[it].begin(), per[it].end());
        max_per_item = std::max(max_per_item, (int)per[it].size());
        if (it % kz == kz - 1) max_per_column = std::max(max_per_column, (int)all.size() - off[it - (kz - 1)]);
    }
    off[items] = (int)all.size();
}

fd_status fused_upload(const std::vector<SrcEntry> &all, const std::vector<int> &off, cudaStream_t st,
                       SparseFused &fused, void *&mem_out)
{
    const size_t b_src = (sizeof(SrcEntry) * all.size() + 15) / 16 * 16;
    const size_t b_off = sizeof(int) * off.size();
    unsigned char *mem = nullptr;
    if (cudaMalloc((void **)&mem, b_src + b_off + 16) != cudaSuccess) return set_error(FD_ERR_NOMEM, "fused sources");
    mem_out = mem;
    cudaError_t e = cudaMemcpyAsync(mem, all.data(), sizeof(SrcEntry) * all.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(mem + b_src, off.data(), b_off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fused sources: %s", cudaGetErrorString(e));
    fused.src = (const SrcEntry *)mem;
    fused.src_off = (const int *)(mem + b_src);
    return FD_OK;
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
    plan.src_cap_col = 0;
    if (!plan.ready) return FD_OK;
    const TileArgs &a = plan.args;
    const int M = plan.M;
    plan.smem = tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, 0);
    if (!src || src->npoint <= 0) return FD_OK;
    std::vector<SrcEntry> all;
    std::vector<int> off;
    int max_s = 0, max_col = 0;
    // one list per CTA (tile column and d0 chunk): a chunk stages only the
    // corners of its own planes
    fused_corner_lists(a, a.kz, src, all, off, max_s, max_col);
    // The CTA's corners are staged in shared memory.  Staging them must
    // keep the CTAs per SM the tiling places (a second wave costs far more
    // than the atomic injection kernel: a receiver lattice injected by the
    // adjoint puts thousands of corners in one tile column), lowering the
    // prefetch depth if that is what it takes; else injection keeps its own
    // kernel.
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ctas = (long long)a.k1 * a.k2 * a.kz;
    const int need = std::min<int>(tma_occupancy(M, plan.stages, plan.threads, plan.smem),
                                   (int)((ctas + sms - 1) / sms));
    int P = plan.stages;
    for (; P >= kMinStages; P--) {
        const size_t with = tma_smem_bytes(M, P, a.rows_max, a.n0, max_s);
        if (with <= plan.smem_max && tma_occupancy(M, P, plan.threads, with) >= need) break;
    }
    if (P < kMinStages) return FD_OK;
    plan.stages = P;
    fd_status s = fused_upload(all, off, st, plan.fused, plan.fused_mem);
    if (s != FD_OK) return s;
    plan.has_src = true;
    plan.src_cap = max_s;
    plan.src_cap_col = max_col;
    plan.smem = tma_smem_bytes(M, plan.stages, a.rows_max, a.n0, plan.src_cap);
    return FD_OK;
}

void tma_plan_tiling(const TmaPlan &plan, int *rows, int *stages, int *ctas)
{
    *rows = plan.ready ? plan.args.rows_max : 0;
    *stages = plan.ready ? plan.stages : 0;
    *ctas = plan.ready ? plan.args.k1 * plan.args.k2 * plan.args.kz : 0;
}

int tma_occupancy(int M, int P, int threads, size_t smem)
{
    int occ = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (M * 8 + P) {
#define CASE(MM, PP)                                                                                      \
    case MM * 8 + PP:                                                                                     \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, acoustic_tma_kernel<MM, PP, false>, threads, \
                                                          smem);                                          \
        break;
#define CASES(MM) CASE(MM, 2) CASE(MM, 3) CASE(MM, 4)
        CASES(1) CASES(2) CASES(3) CASES(4) CASES(5) CASES(6) CASES(7) CASES(8)
#undef CASES
#undef CASE
    }
    return e == cudaSuccess ? occ : 0;
}

static cudaError_t launch_maps(const TmaPlan &plan, int M, const Coef &cf, const CUtensorMap &map_cur,
                               const CUtensorMap &map_prev, float *out, int *status, const float *src_row,
                               cudaStream_t st, const ImagingArgs &img = ImagingArgs())
{
    dim3 grid((unsigned)(plan.args.k1 * plan.args.k2 * plan.args.kz));
    dim3 block((unsigned)plan.threads);
    const float *srow = plan.has_src ? src_row : nullptr;
    const int key = M * 8 + plan.stages;
    const bool image = img.grad != nullptr;
    switch (key) {
#define CASE(MM, PP)                                                                                      \
    case MM * 8 + PP:                                                                                     \
        if (image)                                                                                        \
            acoustic_tma_kernel<MM, PP, true><<<grid, block, plan.smem, st>>>(                            \
                map_cur, map_prev, plan.c_tile, plan.d_tile, out, plan.args, cf, status, plan.fused.src,  \
                plan.fused.src_off, srow, plan.src_cap, img);                                             \
        else                                                                                              \
            acoustic_tma_kernel<MM, PP, false><<<grid, block, plan.smem, st>>>(                           \
                map_cur, map_prev, plan.c_tile, plan.d_tile, out, plan.args, cf, status, plan.fused.src,  \
                plan.fused.src_off, srow, plan.src_cap, img);                                             \
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

cudaError_t launch_acoustic_tma_imaging(const TmaPlan &plan, int M, const Coef &cf, int cur, int *status,
                                        const float *src_row, const ImagingArgs &img, cudaStream_t st)
{
    const int prev = cur ^ 1;
    return launch_maps(plan, M, cf, plan.u_halo[cur], plan.u_tile[prev], plan.slot[prev], status, src_row, st, img);
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
