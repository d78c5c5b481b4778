// Many shots in one launch per time step (fd_batch_*).
//
// A batch is a set of 3D acoustic operators -- one per shot, each on its own
// grid (e.g. a subgrid window of a large model) -- that advance together.
// Every time step is one launch of a persistent kernel: each CTA's producer
// warp takes work items from one list as the CTA's ring has room, and the CTA
// sweeps tile columns of any shot with the single-grid kernel's producer and
// consumer code (k_sweep.cuh: ring positions run on across columns, so the
// pipeline does not drain between them), or gathers receivers of any shot
// from u^n in global memory (no CTA writes u^n during a step).  The list is
// in decreasing cost (plane-rows), taken longest-processing-time-first at
// run time, so shots of uneven sizes fill the GPU together.  The whole time
// loop can be captured once as a CUDA graph and replayed.
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

// True when a column of this shot fits the launch: its per-plane starts and
// nsrc corners within the staged room.  Producer and compute warps decide it
// alike, from the same values.
template <int M, int P>
__device__ __forceinline__ bool column_fits(int rows_max, int src_cap, int n0, int nsrc)
{
    return nsrc <= src_cap && tma_smem_layout(M, P, rows_max, src_cap, n0).end <= (size_t)dynamic_smem_bytes();
}

// The persistent many-shot step.  Items (sorted by decreasing cost) are taken
// from a global counter by the producer warp's lane as soon as the CTA's ring
// has room: it publishes each item in one of two shared slots and, for a
// tile column, issues the column's copies behind the previous column's, so
// the pipeline does not drain between columns.  The compute warps take the
// items in the same order: a column is swept by ws_consume_column (the
// single-grid kernel's arithmetic), a receiver chunk interpolated.  Item
// slot t % 2 carries the CTA's t-th item: "full" when the lane wrote it,
// "empty" when every compute thread has read it.
template <int M, int P>
__global__ void __launch_bounds__(16 * kMaxRowsTiled + 32, 1)
    acoustic_batch_kernel(const ShotDesc *__restrict__ shots, const BatchItem *__restrict__ items, const int nitems,
                          int *next_item, const Coef cf, const int rows_max, const int src_cap, const long long n,
                          const int cur, int *status)
{
    if (*reinterpret_cast<volatile int *>(status) != 0) return;
    // everything but the per-plane starts (checked per column)
    if (!smem_fits<M, P>(rows_max, src_cap, 0, status)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const SweepSmem sm = carve_smem<M, P>(smem_raw, rows_max, src_cap);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int compute_warps = (int)(blockDim.x >> 5) - 1;
    const int nthreads = 32 * compute_warps;
    init_barriers_ws<M, P>(sm, (unsigned)compute_warps);
    constexpr int kItem = ws_item_bar<M, P>();
    auto ITEM_FULL = [&](int s) { return smem_addr(&sm.bars[kItem + s]); };
    auto ITEM_EMPTY = [&](int s) { return smem_addr(&sm.bars[kItem + 2 + s]); };
    // a whole column's corners: the runs of all its d0 chunks, one after another
    auto corners = [&](const ShotDesc *sd, int tile, int &s0) {
        s0 = 0;
        if (!sd->src) return 0;
        s0 = sd->src_off[tile * sd->a.kz];
        return sd->src_off[(tile + 1) * sd->a.kz] - s0;
    };

    if (warp == compute_warps) {
        if (lane == 0) {
            unsigned nu = 0, na = 0;
            bool ok = true;
            for (unsigned t = 0;; t++) {
                const int k = atomicAdd(next_item, 1);
                const int s = (int)(t & 1);
                if (t >= 2 && !mbar_wait_flag(ITEM_EMPTY(s), ((t >> 1) - 1) & 1, sm.abort)) {
                    ok = false;
                    break;
                }
                sm.items[s] = k;
                mbar_arrive_cta(ITEM_FULL(s));
                if (k >= nitems) break;
                const BatchItem it = items[k];
                if (it.kind != 0) continue;
                const ShotDesc *sd = shots + it.shot;
                int s0;
                if (!column_fits<M, P>(rows_max, src_cap, sd->a.n0, corners(sd, it.lo, s0))) {
                    // more than the launch staged room for: nothing of this
                    // column is issued
                    atomicCAS(status, 0, (int)FD_ERR_LAYOUT);
                    ok = false;
                    break;
                }
                if (!ws_produce_column<M, P>(&sd->u_halo[cur], &sd->u_tile[cur ^ 1], &sd->c_tile, &sd->d_tile,
                                             sd->a, it.lo, 0, sd->a.n0, sm, nu, na)) {
                    ok = false;
                    break;
                }
            }
            if (!ok || *sm.abort) ws_drain<M, P>(sm, nu, na, status);
        }
        __syncwarp();
        return;
    }

    // compute warps: every decision to leave is taken by all of them alike
    // (named_barrier_or), so none waits at a barrier the others have left
    unsigned ub = 0, ab = 0;
    for (unsigned t = 0;; t++) {
        const int s = (int)(t & 1);
        const bool got = mbar_wait_flag(ITEM_FULL(s), (t >> 1) & 1, sm.abort);
        const int k = got ? sm.items[s] : nitems;
        if (got) mbar_arrive_cta(ITEM_EMPTY(s));
        if (named_barrier_or(1, nthreads, !got)) {
            if (threadIdx.x == 0) {
                *sm.abort = 1;
                atomicCAS(status, 0, (int)FD_ERR_TIMEOUT);
            }
            break;
        }
        if (k >= nitems) break;
        const BatchItem it = items[k];
        const ShotDesc *sd = shots + it.shot;
        if (it.kind == 0) {
            int s0;
            const int nsrc = corners(sd, it.lo, s0);
            if (!column_fits<M, P>(rows_max, src_cap, sd->a.n0, nsrc)) break;  // the producer records it
            const float *src_row = sd->src ? sd->src_trace + n * sd->src_stride : nullptr;
            stage_sources(sd->src + s0, nsrc, sd->a.n0, sm, nthreads, [&] { named_barrier(1, nthreads); });
            const bool ok = ws_consume_column<M, P, false>(sd->a, cf, it.lo, 0, sd->a.n0, sd->slot[cur ^ 1], nsrc,
                                                           src_row, sm, ub, ab, status, ImagingArgs());
            ub += (unsigned)(sd->a.n0 + 2 * M);
            ab += (unsigned)sd->a.n0;
            // also: every compute thread is done with this column's corners
            if (named_barrier_or(1, nthreads, !ok || *sm.abort)) break;
        } else {
            // rec[n][p] = sum_k w_pk u^n(base_p + off_k), as interpolate_kernel
            const float *u = sd->slot[cur];
            float *row = sd->rec_trace + n * sd->rec_stride;
            for (int p = it.lo + (int)threadIdx.x; p < it.hi; p += nthreads) {
                const int64_t b = sd->rec.base[p];
                const float *w = sd->rec.weight + (int64_t)p * 8;
                float acc = 0.0f;
                for (int c = 0; c < sd->rec.ncorner; c++) acc = fmaf(w[c], u[b + sd->rec.corner_off[c]], acc);
                row[p] = acc;
            }
        }
    }
}

constexpr int kBatchRecChunk = 2048;

// The kernel instance of space order 2M with P stages (null: none).
const void *batch_kernel(int M, int P)
{
    switch (M * 8 + P) {
#define CASE(MM, PP) \
    case MM * 8 + PP: return reinterpret_cast<const void *>(&acoustic_batch_kernel<MM, PP>);
#define CASES(MM) CASE(MM, 2) CASE(MM, 3) CASE(MM, 4)
        CASES(1) CASES(2) CASES(3) CASES(4) CASES(5) CASES(6) CASES(7) CASES(8)
#undef CASES
#undef CASE
    default: return nullptr;
    }
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
        if (p->has_src) src_cap = std::max(src_cap, p->src_cap_col);
    }
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = tma_smem_bytes(M, stages, rows_max, n0_max, src_cap);
    if (smem > (size_t)smem_max) return set_error(FD_ERR_UNSUPPORTED, "batch: %d stages do not fit", stages);
    if (rows_max > kMaxRowsTiled)
        return set_error(FD_ERR_UNSUPPORTED, "batch: tiles of %d rows (at most %d)", rows_max, kMaxRowsTiled);
    const int threads = tma_threads(rows_max);
    const void *kernel = batch_kernel(M, stages);
    if (!kernel) return set_error(FD_ERR_UNSUPPORTED, "batch: space order %d, %d stages", 2 * M, stages);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    // resident CTAs per SM for these threads, registers and shared memory
    int occ = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "batch: kernel configuration: %s", cudaGetErrorString(e));
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
    e = cudaMemcpyAsync(mem, shots.data(), b_shots, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !flat.empty())
        e = cudaMemcpyAsync(mem + b_shots, flat.data(), sizeof(BatchItem) * flat.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return set_error(FD_ERR_CUDA, "batch: upload: %s", cudaGetErrorString(e));
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
