// Tiled (TMA-staged) stencil kernels: plan and launcher.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "fd_internal.h"

namespace fdgb {

constexpr int kTileW = 64;       // tile width along the contiguous axis d2
constexpr int kSideHalo = 8;     // columns loaded on each side of a tile (>= M, keeps x 16-byte aligned)
constexpr int kBoxW = kTileW + 2 * kSideHalo;
// rows (d1) per tile at most: the compute warps plus the producer warp stay
// within 16 warps, so each thread can hold 128 registers
constexpr int kMaxRowsTiled = 30;

// Threads of a single-grid tiled CTA: 16 per tile row (4 points each),
// rounded up to whole warps, plus the producer warp that issues the copies.
inline int tma_threads(int rows_max) { return (16 * rows_max + 31) / 32 * 32 + 32; }

// Geometry handed to the tiled kernel.
struct TileArgs {
    int n0, n1, n2;      // interior extents
    long long s0, s1;    // element strides of d0 and d1
    int k1, k2;          // tiles along d1 (balanced strips) and d2 (64 wide)
    int kz;              // chunks of d0 (balanced), each swept by its own CTA
    int stall_plane;     // test hook: tile 0 never receives this u^n plane (-1: off)
    int rows_max;        // tallest strip
    int box_h;           // rows of a haloed tile: rows_max + 2M
};

// One injected corner: its d0 plane, row and column inside the owning tile,
// the source's trace column and the linear weight.
struct SrcEntry {
    int z;
    int r;
    int x;
    int p;
    float w;
};

// The imaging condition of the adjoint-state gradient, fused into a step:
// grad += scale * w * (u0 - 2 u1 + u2) at every point the step writes, w the
// value it writes there (u0, u1, u2, grad in the slot layout).  Off when
// grad is null.
struct ImagingArgs {
    const float *u0 = nullptr;
    const float *u1 = nullptr;
    const float *u2 = nullptr;
    float *grad = nullptr;
    float scale = 0.0f;
};

// The thread of a tiled sweep that owns an injected corner: its row and
// group of 4 columns (the order of a plane's entries after the plane).
__host__ __device__ inline int src_owner_key(const SrcEntry &e) { return e.r * (kTileW / 4) + (e.x >> 2); }

// Device table of the fused source injection, sorted by (tile, plane), with
// per-tile ranges.
struct SparseFused {
    const SrcEntry *src = nullptr;
    const int *src_off = nullptr;   // [tiles + 1]
};

// Host view of a sparse object's interpolation table.
struct SparseHostView {
    int npoint;
    const int64_t *base;
    const float *weight;  // [npoint][8]
};

struct TmaPlan {
    bool ready = false;
    int force_rows = 0;    // > 0: tile height chosen by the caller (autotuner)
    int force_stages = 0;  // > 0: prefetch depth chosen by the caller
    int stall_plane = -1;  // test hook (TileArgs::stall_plane), kept across rebuilds
    int kind = 0;
    int M = 0;
    int stages = 0;      // prefetch depth P
    TileArgs args{};
    int threads = 0;
    size_t smem = 0;       // dynamic shared memory of a launch
    size_t smem_max = 0;   // the device's opt-in limit
    CUtensorMap u_halo[2];   // slot s of u, haloed box (kBoxW x box_h x 1)
    CUtensorMap u_tile[2];   // slot s of u, tile box (kTileW x rows_max x 1)
    CUtensorMap c_tile, d_tile;
    float *slot[2] = {nullptr, nullptr};
    // fused receiver interpolation / source injection (library-owned)
    SparseFused fused;
    void *fused_mem = nullptr;
    bool has_src = false;
    int src_cap = 0;      // injected corners a CTA (tile column, d0 chunk) stages in shared memory
    int src_cap_col = 0;  // the same for a whole tile column (the batched kernel's items)
    // tensor maps of buffers other than the two slots (out-of-place steps)
    struct CachedMap {
        const void *ptr;
        bool halo;
        CUtensorMap map;
    };
    std::vector<CachedMap> cache;
};

// Build the plan for an operator (3D acoustic only; other cases leave
// plan.ready false and use the plain kernels).
fd_status tma_plan_build(TmaPlan &plan, int kind, int space_order, const Geom &g,
                         float *const slot[2], float *c, float *d);
void tma_plan_release(TmaPlan &plan, cudaStream_t st);

// Tile height and prefetch depth of a built plan (for reporting).
void tma_plan_tiling(const TmaPlan &plan, int *rows, int *stages, int *ctas);


// One acoustic step between arbitrary buffers: reads u_cur (haloed) and
// u_prev, writes u_next (may equal u_prev).  Tensor maps are encoded on first
// use of a buffer and cached.
cudaError_t launch_acoustic_tma_buffers(TmaPlan &plan, int M, const Coef &cf, const float *u_cur,
                                        const float *u_prev, float *u_next, int *status,
                                        const float *src_row, cudaStream_t st);

// Build the fused source-injection table of the plan (src may be null or
// empty); leaves has_src false when the per-tile lists do not fit.
fd_status tma_sparse_build(TmaPlan &plan, const SparseHostView *src, cudaStream_t st);

// One acoustic step: reads slot `cur` (u^n) and slot cur^1 (u^{n-1}),
// overwrites slot cur^1 with u^{n+1}; adds c Q^T src_row when src_row is
// given and the plan fuses the sources.
cudaError_t launch_acoustic_tma(const TmaPlan &plan, int M, const Geom &g, const Coef &cf,
                                int cur, int *status, const float *src_row, cudaStream_t st);
// The same step with the imaging condition fused (img.grad not null).  Only
// valid when the step's sources are fused too (plan.has_src, or no sources):
// the imaged value must be the final one.
cudaError_t launch_acoustic_tma_imaging(const TmaPlan &plan, int M, const Coef &cf, int cur, int *status,
                                        const float *src_row, const ImagingArgs &img, cudaStream_t st);

// CTAs of the tiled kernel of half-width M and depth P resident per SM with
// `threads` threads and `smem` bytes of dynamic shared memory (0 if none).
int tma_occupancy(int M, int P, int threads, size_t smem);

// Tensor map of a 3D field of the tiling `a` with a box of box_w x box_h x 1.
fd_status tma_encode_3d(CUtensorMap *map, float *base, const TileArgs &a, int box_w, int box_h);

// Injected corners of the point set `src` per (tile t, d0 chunk c) of the
// tiling `a` cut into kz chunks, each list sorted by plane (then by owning
// thread): all[off[t kz + c] .. off[t kz + c + 1]) belong to that CTA, and
// all[off[t kz] .. off[(t + 1) kz]) to the whole tile column.  max_per_item
// and max_per_column: the longest of each.
void fused_corner_lists(const TileArgs &a, int kz, const SparseHostView *src, std::vector<SrcEntry> &all,
                        std::vector<int> &off, int &max_per_item, int &max_per_column);
// Copy the lists to one device allocation (mem_out, freed by the caller).
fd_status fused_upload(const std::vector<SrcEntry> &all, const std::vector<int> &off, cudaStream_t st,
                       SparseFused &fused, void *&mem_out);

// ---- two time steps per sweep (k_pair.cu) ---------------------------------

// Plan of the two-step kernel: one CTA per tile column (kz = 1), every column
// resident at once (cooperative launch), progress flags per column.
struct PairPlan {
    bool ready = false;
    int force_rows = 0;      // > 0: tile height chosen by the caller
    int M = 0;
    int stages = 0;          // prefetch depth of the u^n ring
    TileArgs args{};
    int threads = 0;
    size_t smem = 0, smem_max = 0;
    CUtensorMap u_halo[2];   // slot s of u, haloed box
    CUtensorMap u_tile[2];   // slot s of u, tile box
    CUtensorMap c_tile, d_tile;
    float *slot[2] = {nullptr, nullptr};
    SparseFused fused;
    void *fused_mem = nullptr;
    bool has_src = false;
    int src_cap = 0;
    int *progress = nullptr;  // [k1 * k2] planes of u^{n+1} written, per column
};

// Build the plan (3D acoustic, SO 4..8 only; otherwise ready stays false).
fd_status pair_plan_build(PairPlan &plan, int space_order, const Geom &g, float *const slot[2], float *c, float *d);
// Build its fused source table; false in has_src when sources exist but the
// per-tile lists do not fit (the operator then steps one at a time).
fd_status pair_sparse_build(PairPlan &plan, const SparseHostView *src, cudaStream_t st);
void pair_plan_release(PairPlan &plan, cudaStream_t st);
// Two steps: slot b holds u^n and slot b^1 u^{n-1}; afterwards slot b^1
// holds u^{n+1} and slot b u^{n+2}.  src_row1 / src_row2 are the source
// rows of the two steps (null: none).
cudaError_t launch_acoustic_pair(const PairPlan &plan, const Coef &cf, int b, int *status, const float *src_row1,
                                 const float *src_row2, cudaStream_t st);

// ---- many shots per launch (k_batch.cu) ----------------------------------

struct ShotDesc;
struct BatchItem;

struct BatchPlan {
    int M = 0, P = 0, rows_max = 0, src_cap = 0, nctas = 0, threads = 0;
    size_t smem = 0;
    Coef cf{};
    ShotDesc *d_shots = nullptr;
    BatchItem *d_items = nullptr;
    int *d_next = nullptr;   // next item to take (reset before every launch)
    int nitems = 0;
};

// Build the device tables of a batch from the shots' tiled plans (all of the
// same space order and coefficients), their receivers and traces.
fd_status batch_plan_build(BatchPlan &bp, const std::vector<const TmaPlan *> &plans,
                           const std::vector<const SparseDev *> &recs, const std::vector<float *> &rec_traces,
                           const std::vector<long long> &rec_strides, const std::vector<const float *> &src_traces,
                           const std::vector<long long> &src_strides, const Coef &cf, int stages,
                           cudaStream_t st);
void batch_plan_release(BatchPlan &bp);
// One time step n of every shot: reads slot `cur`, writes slot cur^1.
cudaError_t launch_batch(const BatchPlan &bp, long long n, int cur, int *status, cudaStream_t st);

}  // namespace fdgb
