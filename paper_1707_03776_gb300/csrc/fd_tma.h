// Tiled (TMA-staged) stencil kernels: plan and launcher.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "fd_internal.h"

namespace fdgb {

constexpr int kTileW = 64;       // tile width along the contiguous axis d2
constexpr int kSideHalo = 8;     // columns loaded on each side of a tile (>= M, keeps x 16-byte aligned)
constexpr int kBoxW = kTileW + 2 * kSideHalo;
constexpr int kMaxRows = 32;     // rows (d1) per tile at most

// Geometry handed to the tiled kernel.
struct TileArgs {
    int n0, n1, n2;      // interior extents
    long long s0, s1;    // element strides of d0 and d1
    int k1, k2;          // tiles along d1 (balanced strips) and d2 (64 wide)
    int rows_max;        // tallest strip
    int box_h;           // rows of a haloed tile: rows_max + 2M
};

struct TmaPlan {
    bool ready = false;
    int kind = 0;
    int M = 0;
    int stages = 0;      // prefetch depth P
    TileArgs args{};
    int threads = 0;
    size_t smem = 0;
    CUtensorMap u_halo[2];   // slot s of u, haloed box (kBoxW x box_h x 1)
    CUtensorMap u_tile[2];   // slot s of u, tile box (kTileW x rows_max x 1)
    CUtensorMap c_tile, d_tile;
    float *slot[2] = {nullptr, nullptr};
};

// Build the plan for an operator (3D acoustic only; other cases leave
// plan.ready false and use the plain kernels).
fd_status tma_plan_build(TmaPlan &plan, int kind, int space_order, const Geom &g,
                         float *const slot[2], float *c, float *d);
void tma_plan_release(TmaPlan &plan);

// One acoustic step: reads slot `cur` (u^n) and slot cur^1 (u^{n-1}),
// overwrites slot cur^1 with u^{n+1}.
cudaError_t launch_acoustic_tma(const TmaPlan &plan, int M, const Geom &g, const Coef &cf,
                                int cur, int *status, cudaStream_t st);

}  // namespace fdgb
