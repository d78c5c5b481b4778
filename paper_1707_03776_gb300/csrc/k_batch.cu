// Many shots in one launch per time step (fd_batch_*).
//
// A batch is a set of 3D acoustic operators -- one per shot, each on its own
// grid (e.g. a subgrid window of a large model) -- that advance together.
// Every time step is one launch of a persistent kernel: each CTA walks a list
// of work items, sweeping tile columns of any shot with the same column sweep
// as the single-grid kernel (k_sweep.cuh: ring slots and mbarrier phases run
// on across columns), and gathering receivers of any shot from u^n in global
// memory (no CTA writes u^n during a step).  Items are spread over the CTAs
// by longest-processing-time-first on their cost in plane-rows, so shots of
// uneven sizes fill the GPU together.  The whole time loop can be captured
// once as a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <queue>
#include <vector>

#include "fd_internal_host.h"
#include "fd_tma.h"
#include "k_sweep.cuh"

namespace fdgb {

// Per-shot state the batch kernel reads (128-byte aligned, as its tensor maps
// are).
struct alignas(128) ShotDesc {
    CUtensorMap u_halo[2];
    CUtensorMap u_tile[2];
    CUtensorMap c_tile;
    CUtensorMap d_tile;
    TileArgs a;
    float *slot[2];
    const SrcEntry *src;       // fused injection table (null: no sources)
    const int *src_off;
    const float *src_trace;    // row n at src_trace + n * src_stride
    long long src_stride;
    SparseDev rec;             // receivers (npoint may be 0)
    float *rec_trace;
    long long rec_stride;
};

// kind 0: sweep tile column `lo` of shot; kind 1: receivers [lo, hi) of shot.
struct BatchItem {
    int kind;
    int shot;
    int lo;
    int hi;
};

namespace {

using namespace tile_dev;

template <int M, int P>
__global__ void __launch_bounds__(16 * kMaxRows, 1)
    acoustic_batch_kernel(const ShotDesc *__restrict__ shots, const BatchItem *__restrict__ items, const int nitems,
                          int *next_item, const Coef cf, const int rows_max, const int src_cap, const long long n,
                          const int cur, int *status)
{
    if (*reinterpret_cast<volatile int *>(status) != 0) return;
    // everything but the per-plane starts (checked per shot below)
    if (!smem_fits<M, P>(rows_max, src_cap, 0, status)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const SweepSmem sm = carve_smem<M, P>(smem_raw, rows_max, src_cap);
    init_barriers<M, P>(sm);
    unsigned it_u = 0, it_a = 0;
    // items are sorted by decreasing cost; each CTA takes the next one as
    // soon as it is free (longest processing time first, balanced at run time)
    for (;;) {
        if (threadIdx.x == 0) *sm.item = atomicAdd(next_item, 1);
        __syncthreads();
        const int k = *sm.item;
        __syncthreads();
        if (k >= nitems) break;
        const BatchItem it = items[k];
        const ShotDesc *sd = shots + it.shot;
        if (it.kind == 0) {
            const TileArgs a = sd->a;
            if (!smem_fits<M, P>(rows_max, src_cap, a.n0, status)) return;
            const float *src_row = nullptr;
            int s0 = 0, nsrc = 0;
            if (sd->src) {
                src_row = sd->src_trace + n * sd->src_stride;
                s0 = sd->src_off[it.lo];
                nsrc = sd->src_off[it.lo + 1] - s0;
            }
            if (nsrc > src_cap) {
                // more corners than the launch staged room for (no copies
                // are in flight between columns)
                if (threadIdx.x == 0) atomicExch(status, (int)FD_ERR_LAYOUT);
                return;
            }
            if (!sweep_column<M, P>(&sd->u_halo[cur], &sd->u_tile[cur ^ 1], &sd->c_tile, &sd->d_tile,
                                    sd->slot[cur ^ 1], a, cf, it.lo, 0, a.n0, sd->src + s0, nsrc, src_row, sm, it_u,
                                    it_a, status))
                return;
        } else {
            // rec[n][p] = sum_k w_pk u^n(base_p + off_k), as interpolate_kernel
            const float *u = sd->slot[cur];
            float *row = sd->rec_trace + n * sd->rec_stride;
            for (int p = it.lo + (int)threadIdx.x; p < it.hi; p += blockDim.x) {
                const int64_t b = sd->rec.base[p];
                const float *w = sd->rec.weight + (int64_t)p * 8;
                float s = 0.0f;
                for (int c = 0; c < sd->rec.ncorner; c++) s = fmaf(w[c], u[b + sd->rec.corner_off[c]], s);
                row[p] = s;
            }
        }
    }
}

constexpr int kBatchRecChunk = 2048;

template <int M>
cudaError_t batch_configure(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(acoustic_batch_kernel<M, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(acoustic_batch_kernel<M, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(acoustic_batch_kernel<M, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    return e;
}

}  // namespace

fd_status batch_plan_build(BatchPlan &bp, const std::vector<const TmaPlan *> &plans,
                           const std::vector<const SparseDev *> &recs, const std::vector<float *> &rec_traces,
                           const std::vector<long long> &rec_strides, const std::vector<const float *> &src_traces,
                           const std::vector<long long> &src_strides, const Coef &cf, int stages, cudaStream_t st)
{
    const int nshots = (int)plans.size();
    const int M = plans[0]->M;
    int rows_max = 0, src_cap = 0, n0_max = 0;
    for (const TmaPlan *p : plans) {
        rows_max = std::max(rows_max, p->args.rows_max);
        n0_max = std::max(n0_max, p->args.n0);
        if (p->has_src) src_cap = std::max(src_cap, p->src_cap);
    }
    int dev = 0, sms = 0, smem_max = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const size_t smem = tma_smem_bytes(M, stages, rows_max, n0_max, src_cap);
    if (smem > (size_t)smem_max) return set_error(FD_ERR_UNSUPPORTED, "batch: %d stages do not fit", stages);
    const int threads = 16 * rows_max;
    int occ = std::min((int)((size_t)smem_sm / (smem + 1024)), 2048 / threads);
    if (occ < 1) return set_error(FD_ERR_UNSUPPORTED, "batch: tiles do not fit on an SM");
    const int nctas = sms * occ;

    // work items and their costs (plane-rows; a receiver costs ~1/128 of one)
    std::vector<BatchItem> items;
    std::vector<double> cost;
    for (int s = 0; s < nshots; s++) {
        const TileArgs &a = plans[s]->args;
        for (int t = 0; t < a.k1 * a.k2; t++) {
            const int strip = t / a.k2;
            const int rows = (int)((int64_t)(strip + 1) * a.n1 / a.k1) - (int)((int64_t)strip * a.n1 / a.k1);
            items.push_back({0, s, t, 0});
            cost.push_back((double)a.n0 * (rows + 0.5 * M) + 2.0 * M * rows);
        }
        const int nrec = recs[s] ? recs[s]->npoint : 0;
        for (int lo = 0; lo < nrec; lo += kBatchRecChunk) {
            const int hi = std::min(nrec, lo + kBatchRecChunk);
            items.push_back({1, s, lo, hi});
            cost.push_back((hi - lo) / 128.0);
        }
    }
    // one list in decreasing cost (receiver chunks, the cheapest, last); the
    // kernel's CTAs take items from it in order as they become free
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<BatchItem> flat;
    flat.reserve(order.size());
    for (int i : order) flat.push_back(items[i]);

    std::vector<ShotDesc> shots(nshots);
    for (int s = 0; s < nshots; s++) {
        const TmaPlan *p = plans[s];
        ShotDesc &d = shots[s];
        std::memset(&d, 0, sizeof d);
        d.u_halo[0] = p->u_halo[0];
        d.u_halo[1] = p->u_halo[1];
        d.u_tile[0] = p->u_tile[0];
        d.u_tile[1] = p->u_tile[1];
        d.c_tile = p->c_tile;
        d.d_tile = p->d_tile;
        d.a = p->args;
        d.slot[0] = p->slot[0];
        d.slot[1] = p->slot[1];
        if (p->has_src && src_traces[s]) {
            d.src = p->fused.src;
            d.src_off = p->fused.src_off;
            d.src_trace = src_traces[s];
            d.src_stride = src_strides[s];
        }
        if (recs[s]) {
            d.rec = *recs[s];
            d.rec_trace = rec_traces[s];
            d.rec_stride = rec_strides[s];
        }
    }
    const size_t b_shots = sizeof(ShotDesc) * nshots;
    const size_t b_items = (sizeof(BatchItem) * std::max<size_t>(flat.size(), 1) + 255) / 256 * 256;
    unsigned char *mem = nullptr;
    if (cudaMalloc((void **)&mem, b_shots + b_items + sizeof(int)) != cudaSuccess)
        return set_error(FD_ERR_NOMEM, "batch: device tables");
    cudaError_t e = cudaMemcpyAsync(mem, shots.data(), b_shots, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !flat.empty())
        e = cudaMemcpyAsync(mem + b_shots, flat.data(), sizeof(BatchItem) * flat.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return set_error(FD_ERR_CUDA, "batch: upload: %s", cudaGetErrorString(e));
    }
    switch (M) {
#define CASE(MM) \
    case MM: e = batch_configure<MM>((size_t)smem_max); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) {
        cudaFree(mem);
        return set_error(FD_ERR_CUDA, "batch: kernel configuration: %s", cudaGetErrorString(e));
    }
    bp.M = M;
    bp.P = stages;
    bp.rows_max = rows_max;
    bp.src_cap = src_cap;
    bp.nctas = nctas;
    bp.threads = threads;
    bp.smem = smem;
    bp.cf = cf;
    bp.d_shots = (ShotDesc *)mem;
    bp.d_items = (BatchItem *)(mem + b_shots);
    bp.d_next = (int *)(mem + b_shots + b_items);
    bp.nitems = (int)flat.size();
    return FD_OK;
}

void batch_plan_release(BatchPlan &bp)
{
    if (bp.d_shots) cudaFree(bp.d_shots);
    bp.d_shots = nullptr;
    bp.d_items = nullptr;
    bp.d_next = nullptr;
    bp.nitems = 0;
}

cudaError_t launch_batch(const BatchPlan &bp, long long n, int cur, int *status, cudaStream_t st)
{
    cudaError_t e0 = cudaMemsetAsync(bp.d_next, 0, sizeof(int), st);
    if (e0 != cudaSuccess) return e0;
    const int key = bp.M * 8 + bp.P;
    switch (key) {
#define CASE(MM, PP)                                                                                          \
    case MM * 8 + PP:                                                                                         \
        acoustic_batch_kernel<MM, PP><<<bp.nctas, bp.threads, bp.smem, st>>>(                                 \
            bp.d_shots, bp.d_items, bp.nitems, bp.d_next, bp.cf, bp.rows_max, bp.src_cap, n, cur, status);   \
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

}  // namespace fdgb
