// Device side of the tiled acoustic kernels: PTX helpers and the sweep of
// one tile column, shared by the single-grid kernel (k_tma.cu) and the
// batched many-shot kernel (k_batch.cu).
//
// A tile column is rows [row0, row0+rows) of d1 and 64 columns of d2 of one
// grid, swept over every d0 plane:
//   * one TMA box brings the haloed u^n tile (64+16 columns, rows+2M rows)
//     into a ring of shared-memory planes; the zero halo around the grid is
//     the TMA out-of-bounds fill, so no halo is stored in HBM;
//   * three TMA boxes bring u^{n-1}, c = dt^2/m and d = dt*eta/m of the plane
//     being finished into a second ring;
//   * every thread owns 4 consecutive d2 points of one row, keeps the 2M+1
//     centre values along d0 in a register queue, reads the d1/d2 neighbours
//     of the plane M behind the newest from shared memory, adds the source
//     injection of the corners it owns and writes u^{n+1} with 128-bit stores.
// One lane of a producer warp issues the copies P planes ahead on mbarriers
// with transaction counts, into slots the compute threads hand back; every
// wait is bounded by the global timer and, when it gives up, the CTA records
// FD_ERR_TIMEOUT in the status word and leaves after draining its own copies.
#pragma once

#include "fd_tma.h"

namespace fdgb {

namespace tile_dev {

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

__device__ __forceinline__ void mbar_arrive_cta(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

// Wait for phase `parity` of a barrier until the globaltimer passes
// `deadline` (a barrier that has already completed returns at once).
__device__ __forceinline__ bool mbar_wait_until(uint32_t bar, uint32_t parity, unsigned long long deadline)
{
    while (!mbar_try_wait(bar, parity))
        if (global_ns() > deadline) return false;
    return true;
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

// Byte offsets of the areas of a tiled CTA's dynamic shared memory: the u^n
// ring, the aux ring, the mbarriers, the abort flag and the batched kernel's
// two work-item slots (16 bytes), then src_cap
// injected corners of the tile and their n0 + 1 per-plane starts.  Both the
// size a launch requests and the carve in the kernel come from here.
struct SmemLayout {
    size_t aux, bars, abort, src, sstart, end;
};

__host__ __device__ inline SmemLayout tma_smem_layout(int M, int P, int rows_max, int src_cap, int n0)
{
    const int NU = M + 1 + P, NA = P + 1;
    SmemLayout l;
    l.aux = sizeof(float) * (size_t)NU * ring_plane_floats(rows_max + 2 * M);
    l.bars = l.aux + sizeof(float) * (size_t)NA * 3 * rows_max * kTileW;
    l.abort = l.bars + sizeof(unsigned long long) * (size_t)(2 * (NU + NA) + 4);  // full, empty, items
    l.src = l.abort + 16;
    l.sstart = l.src + sizeof(SrcEntry) * (size_t)src_cap;
    l.end = l.sstart + sizeof(int) * (size_t)(n0 + 1);
    return l;
}

// Without the point lists (the part every launch needs).
__host__ __device__ inline size_t tma_smem_core(int M, int P, int rows_max)
{
    return tma_smem_layout(M, P, rows_max, 0, 0).src;
}

__host__ __device__ inline size_t tma_smem_bytes(int M, int P, int rows_max, int n0, int src_cap)
{
    return tma_smem_layout(M, P, rows_max, src_cap, n0).end;
}


// Shared-memory areas of a tiled CTA (sized for the largest column it sweeps).
struct SweepSmem {
    float *ring;                 // NU planes of plane_u floats
    float *aux;                  // NA slots of 3 boxes of plane_a floats
    unsigned long long *bars;    // 2 (NU + NA) + 4 mbarriers
    volatile int *abort;
    volatile int *items;         // batched kernel: two work-item slots (after abort)
    SrcEntry *src;               // the column's injected corners
    int *sstart;                 // per-plane starts into src
    int plane_u, plane_a;
};

__device__ __forceinline__ uint32_t dynamic_smem_bytes()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// True when the launch's dynamic shared memory holds the layout of a CTA with
// these parameters; otherwise records FD_ERR_LAYOUT in the status word (the
// CTA must then return without touching shared memory).
template <int M, int P>
__device__ inline bool smem_fits(int rows_max, int src_cap, int n0, int *status)
{
    if (tma_smem_layout(M, P, rows_max, src_cap, n0).end <= (size_t)dynamic_smem_bytes()) return true;
    if (threadIdx.x == 0) atomicExch(status, (int)FD_ERR_LAYOUT);
    return false;
}

// Carve the dynamic shared memory of a CTA whose columns have at most
// rows_max rows, n0_max planes and src_cap injected corners.
template <int M, int P>
__device__ inline SweepSmem carve_smem(unsigned char *raw, int rows_max, int src_cap)
{
    const SmemLayout l = tma_smem_layout(M, P, rows_max, src_cap, 0);
    SweepSmem sm;
    sm.plane_u = ring_plane_floats(rows_max + 2 * M);
    sm.plane_a = rows_max * kTileW;
    sm.ring = reinterpret_cast<float *>(raw);
    sm.aux = reinterpret_cast<float *>(raw + l.aux);
    sm.bars = reinterpret_cast<unsigned long long *>(raw + l.bars);
    sm.abort = reinterpret_cast<volatile int *>(raw + l.abort);
    sm.items = reinterpret_cast<volatile int *>(raw + l.abort) + 2;
    sm.src = reinterpret_cast<SrcEntry *>(raw + l.src);
    sm.sstart = reinterpret_cast<int *>(raw + l.sstart);
    return sm;
}

// One output plane of a thread's 4 consecutive d2 points (row r, columns
// col0 + 4 qc ..): the Laplacian from the centre plane's haloed tile in
// shared memory (pc: the first point, d1/d2 neighbours around it) and the d0
// queue q, the update, the fused source corners of the plane, the store of
// u^{n+1} and (IMG) the imaging condition from img_cur.  Every tiled sweep
// uses it, so they agree bit for bit.
template <int M, bool IMG>
__device__ __forceinline__ void update_points(const float *__restrict__ pc, const float *__restrict__ pa, int plane_a,
                                              const float4 (&q)[2 * M + 1], const Coef &cf, const TileArgs &a,
                                              int row0, int col0, int r, int qc, int zo, float *__restrict__ out,
                                              int nsrc, const SrcEntry *s_src, const int *s_sstart,
                                              const float *__restrict__ src_row, const ImagingArgs &img,
                                              const float4 (&img_cur)[4])
{
    constexpr int HV = (M + 3) / 4;   // float4 groups on each side of a thread's 4 points
    constexpr int NR = 4 * (2 * HV + 1);
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
        const float4 um4 = *reinterpret_cast<const float4 *>(pa);
        const float4 c4 = *reinterpret_cast<const float4 *>(pa + plane_a);
        const float4 d4 = *reinterpret_cast<const float4 *>(pa + 2 * plane_a);
        const float umv[4] = {um4.x, um4.y, um4.z, um4.w};
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
        const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
        // Laplacian of the 4 points as two pairs, with the packed
        // FP32 instructions (two lanes per issue).  Each lane does
        // the same operations in the same order as the scalar form
        // centre*u, then per k: ax2*(d2 pair) + ax1*(d1 pair) +
        // ax0*(d0 pair), so the result is bitwise unchanged.
        float lapv[4];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int c = 4 * HV + 2 * h;
            float2 lap = __fmul2_rn(make_float2(cf.centre, cf.centre), make_float2(row[c], row[c + 1]));
#pragma unroll
            for (int k = 1; k <= M; k++) {
                const float4 lo = q[M - k];
                const float4 hi = q[M + k];
                // an odd k puts the d2 pair across a 64-bit register
                // boundary: two scalar adds then, not a packed one
                const float2 s2 =
                    (k % 2 == 0)
                        ? __fadd2_rn(make_float2(row[c - k], row[c - k + 1]),
                                     make_float2(row[c + k], row[c + k + 1]))
                        : make_float2(row[c - k] + row[c + k], row[c + 1 - k] + row[c + 1 + k]);
                const float2 s1 = h ? __fadd2_rn(make_float2(cm[k].z, cm[k].w), make_float2(cp[k].z, cp[k].w))
                                    : __fadd2_rn(make_float2(cm[k].x, cm[k].y), make_float2(cp[k].x, cp[k].y));
                const float2 s0 = h ? __fadd2_rn(make_float2(lo.z, lo.w), make_float2(hi.z, hi.w))
                                    : __fadd2_rn(make_float2(lo.x, lo.y), make_float2(hi.x, hi.y));
                lap = __ffma2_rn(make_float2(cf.ax[2][k], cf.ax[2][k]), s2, lap);
                lap = __ffma2_rn(make_float2(cf.ax[1][k], cf.ax[1][k]), s1, lap);
                lap = __ffma2_rn(make_float2(cf.ax[0][k], cf.ax[0][k]), s0, lap);
            }
            lapv[2 * h] = lap.x;
            lapv[2 * h + 1] = lap.y;
        }
        float res[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float u = row[4 * HV + i];
            // 2u - u- + c Lu - d (u - u-) as three explicit FMAs (2u is
            // exact), the same chain in every acoustic kernel
            res[i] = fmaf(-dv[i], u - umv[i], fmaf(cv[i], lapv[i], fmaf(2.0f, u, -umv[i])));
        }
        if (nsrc > 0) {
            // source injection at the corners this thread owns on plane ja
            // (a plane's entries are sorted by owning thread: binary
            // search for this thread's first, then its run)
            float inj0 = 0.f, inj1 = 0.f, inj2 = 0.f, inj3 = 0.f;
            const int s_end = s_sstart[zo + 1];
            const int key = r * (kTileW / 4) + qc;
            int lo = s_sstart[zo], hi = s_end;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (src_owner_key(s_src[mid]) < key) lo = mid + 1; else hi = mid;
            }
            for (int k = lo; k < s_end; k++) {
                const SrcEntry e = s_src[k];
                if (src_owner_key(e) != key) break;
                const float sv = e.w * src_row[e.p];
                const int i = e.x & 3;
                inj0 += (i == 0) ? sv : 0.f;
                inj1 += (i == 1) ? sv : 0.f;
                inj2 += (i == 2) ? sv : 0.f;
                inj3 += (i == 3) ? sv : 0.f;
            }
            res[0] = fmaf(inj0, cv[0], res[0]);
            res[1] = fmaf(inj1, cv[1], res[1]);
            res[2] = fmaf(inj2, cv[2], res[2]);
            res[3] = fmaf(inj3, cv[3], res[3]);
        }
        const long long at = (long long)zo * a.s0 + (long long)(row0 + r) * a.s1 + col0 + 4 * qc;
        float *o = out + at;
        const bool full = col0 + 4 * qc + 3 < a.n2;
        if (full) {
            *reinterpret_cast<float4 *>(o) = make_float4(res[0], res[1], res[2], res[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (col0 + 4 * qc + i < a.n2) o[i] = res[i];
        }
        if constexpr (IMG) {
            // grad += scale * w * (u0 - 2 u1 + u2), the same two FMAs
            // and add as the separate imaging kernel
            if (full) {
                const float4 x0 = img_cur[0], x1 = img_cur[1], x2 = img_cur[2];
                float4 gr = img_cur[3];
                gr.x = fmaf(img.scale * res[0], fmaf(-2.0f, x1.x, x0.x) + x2.x, gr.x);
                gr.y = fmaf(img.scale * res[1], fmaf(-2.0f, x1.y, x0.y) + x2.y, gr.y);
                gr.z = fmaf(img.scale * res[2], fmaf(-2.0f, x1.z, x0.z) + x2.z, gr.z);
                gr.w = fmaf(img.scale * res[3], fmaf(-2.0f, x1.w, x0.w) + x2.w, gr.w);
                *reinterpret_cast<float4 *>(img.grad + at) = gr;
            } else {
                const float x0[4] = {img_cur[0].x, img_cur[0].y, img_cur[0].z, img_cur[0].w};
                const float x1[4] = {img_cur[1].x, img_cur[1].y, img_cur[1].z, img_cur[1].w};
                const float x2[4] = {img_cur[2].x, img_cur[2].y, img_cur[2].z, img_cur[2].w};
                const float gr[4] = {img_cur[3].x, img_cur[3].y, img_cur[3].z, img_cur[3].w};
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (col0 + 4 * qc + i < a.n2)
                        img.grad[at + i] = fmaf(img.scale * res[i], fmaf(-2.0f, x1[i], x0[i]) + x2[i], gr[i]);
            }
        }
}

// Column sweeps with a producer warp.  The CTA's last warp issues the
// copies, P planes ahead, into ring slots that the compute warps hand back
// through "empty" mbarriers (one arrival per compute thread after its last
// read of the slot), so that a compute warp waits only for its own data,
// never for the other warps, and warps may drift up to P planes apart.
// Barriers: full u^n [NU], full aux [NA], empty u^n [NU], empty aux [NA],
// then the batched kernel's work-item slots (full [2], empty [2]).  Every
// wait is bounded; a wait that gives up records FD_ERR_TIMEOUT and raises
// the CTA's abort flag, which every role checks; the producer then drains
// the copies it still owes.
//
// Ring positions: the k-th u^n copy a CTA issues goes to slot k % NU and
// completes phase (k / NU) & 1 of that slot's barriers, the k-th aux copy
// likewise in slot k % NA.  A CTA that sweeps several columns (the batched
// kernel) continues the count from one column to the next, so its pipeline
// never drains between columns.
template <int M, int P>
__host__ __device__ constexpr int ws_item_bar()
{
    return 2 * ((M + 1 + P) + (P + 1));
}

template <int M, int P>
__device__ inline void init_barriers_ws(const SweepSmem &sm, unsigned compute_warps)
{
    constexpr int NU = M + 1 + P, NA = P + 1, kItem = ws_item_bar<M, P>();
    if (threadIdx.x == 0) {
        for (int i = 0; i < NU + NA; i++) mbar_init(smem_addr(&sm.bars[i]), 1);
        for (int i = NU + NA; i < 2 * (NU + NA); i++) mbar_init(smem_addr(&sm.bars[i]), 32 * compute_warps);
        for (int i = 0; i < 2; i++) {
            mbar_init(smem_addr(&sm.bars[kItem + i]), 1);
            mbar_init(smem_addr(&sm.bars[kItem + 2 + i]), 32 * compute_warps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *sm.abort = 0;
    }
    __syncthreads();
}

// Wait for phase `parity`, giving up after kWaitLimitNs or when the abort
// flag is raised.
__device__ __forceinline__ bool mbar_wait_flag(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

// Barrier `id` over the first `nthreads` threads (the compute warps),
// returning whether any of them passed v = true: a decision all of them take
// alike.  Not the .aligned form: threads may arrive from divergent paths.
__device__ __forceinline__ bool named_barrier_or(int id, int nthreads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\t"
        "setp.ne.u32 pi, %1, 0;\n\t"
        "barrier.cta.red.or.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void named_barrier(int id, int nthreads)
{
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Stage a column's injected corners and their per-plane starts (planes
// 0..n0) in shared memory, by threads [0, nthreads), `sync` after each part.
template <class Sync>
__device__ inline void stage_sources(const SrcEntry *__restrict__ src_tab, int nsrc, int n0, const SweepSmem &sm,
                                     int nthreads, Sync sync)
{
    const int tid = threadIdx.x;
    for (int q = tid; q < nsrc * 5; q += nthreads)
        reinterpret_cast<int *>(sm.src)[q] = reinterpret_cast<const int *>(src_tab)[q];
    sync();
    if (nsrc > 0) {
        for (int z = tid; z <= n0; z += nthreads) {
            int lo = 0, hi = nsrc;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sm.src[mid].z < z) lo = mid + 1; else hi = mid;
            }
            sm.sstart[z] = lo;
        }
        sync();
    }
}

// The producer's part of the sweep of output planes [z_lo, z_hi) of tile
// `tile` (one lane): u^n plane j of the column (z = z_lo - M + j) is the
// CTA's u^n copy nu + j, the aux of output plane ja its aux copy na + ja; nu
// and na advance by the copies issued.  False when a wait gave up or the
// abort flag is up (the caller then drains).
template <int M, int P>
__device__ bool ws_produce_column(const CUtensorMap *map_u, const CUtensorMap *map_um, const CUtensorMap *map_c,
                                  const CUtensorMap *map_d, const TileArgs &a, int tile, int z_lo, int z_hi,
                                  const SweepSmem &sm, unsigned &nu, unsigned &na)
{
    constexpr int NU = M + 1 + P, NA = P + 1;
    constexpr int kFullA = NU, kEmptyU = NU + NA, kEmptyA = 2 * NU + NA;
    const int strip = tile / a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int col0 = (tile - strip * a.k2) * kTileW;
    const int J = (z_hi - z_lo) + 2 * M;
    const uint32_t bytes_u = (uint32_t)(kBoxW * a.box_h * sizeof(float));
    const uint32_t bytes_a = (uint32_t)(3 * a.rows_max * kTileW * sizeof(float));
    auto BAR = [&](int i) { return smem_addr(&sm.bars[i]); };
    for (int j = 0; j < J; j++) {
        const unsigned U = nu;
        const int su = (int)(U % NU);
        // the slot's previous copy, U - NU, must have been handed back
        if (U >= NU && !mbar_wait_flag(BAR(kEmptyU + su), ((U / NU) - 1) & 1, sm.abort)) return false;
        mbar_expect_tx(BAR(su), bytes_u);
        // the stall hook arms the barrier but never issues the copy, so the
        // wait for this plane runs out (the failure path under test)
        if (a.stall_plane < 0 || tile != 0 || z_lo - M + j != a.stall_plane)
            tma_load_3d(smem_addr(sm.ring + su * sm.plane_u), map_u, col0 - kSideHalo, row0 - M, z_lo - M + j,
                        BAR(su));
        nu = U + 1;
        if (j >= 2 * M) {
            const unsigned A = na;
            const int sa = (int)(A % NA);
            if (A >= NA && !mbar_wait_flag(BAR(kEmptyA + sa), ((A / NA) - 1) & 1, sm.abort)) return false;
            float *dst = sm.aux + sa * 3 * sm.plane_a;
            const int z = z_lo + (j - 2 * M);
            mbar_expect_tx(BAR(kFullA + sa), bytes_a);
            tma_load_3d(smem_addr(dst), map_um, col0, row0, z, BAR(kFullA + sa));
            tma_load_3d(smem_addr(dst + sm.plane_a), map_c, col0, row0, z, BAR(kFullA + sa));
            tma_load_3d(smem_addr(dst + 2 * sm.plane_a), map_d, col0, row0, z, BAR(kFullA + sa));
            na = A + 1;
        }
    }
    return !*sm.abort;
}

// After a failed wait: raise the abort flag, record FD_ERR_TIMEOUT (unless an
// error is already recorded) and wait, under one shared deadline, for the
// copies possibly still in flight (the last NU u^n and NA aux copies).
template <int M, int P>
__device__ void ws_drain(const SweepSmem &sm, unsigned nu, unsigned na, int *status)
{
    constexpr int NU = M + 1 + P, NA = P + 1;
    *sm.abort = 1;
    atomicCAS(status, 0, (int)FD_ERR_TIMEOUT);
    const unsigned long long deadline = global_ns() + kWaitLimitNs;
    for (unsigned k = nu > NU ? nu - NU : 0; k < nu; k++)
        mbar_wait_until(smem_addr(&sm.bars[k % NU]), (k / NU) & 1, deadline);
    for (unsigned k = na > NA ? na - NA : 0; k < na; k++)
        mbar_wait_until(smem_addr(&sm.bars[NU + k % NA]), (k / NA) & 1, deadline);
}

// The compute warps' part of the same sweep: u^n plane j of the column is
// the CTA's copy ub + j, the aux of output plane ja its aux copy ab + ja (as
// the producer issued them).  Each thread hands every slot back after its
// last read of it: planes j < M and j >= J - M right after they enter the d0
// queue, every other plane after it served as the centre plane (iteration
// j + M), the aux of output plane ja at iteration ja + 2M.  False when a wait
// gave up (FD_ERR_TIMEOUT recorded, abort flag raised) or the flag was up.
// With IMG, the imaging condition of `img` is accumulated at every point
// written, from the value written (sources included).
template <int M, int P, bool IMG>
__device__ bool ws_consume_column(const TileArgs &a, const Coef &cf, int tile, int z_lo, int z_hi,
                                  float *__restrict__ out, int nsrc, const float *__restrict__ src_row,
                                  const SweepSmem &sm, unsigned ub, unsigned ab, int *status,
                                  const ImagingArgs &img)
{
    constexpr int NU = M + 1 + P;     // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;         // aux planes (u^{n-1}, c, d)
    constexpr int kFullA = NU, kEmptyU = NU + NA, kEmptyA = 2 * NU + NA;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int strip = tile / a.k2;
    const int tile2 = tile - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = tile2 * kTileW;
    const int r = tid >> 4;
    const int qc = tid & 15;
    const int J = (z_hi - z_lo) + 2 * M;
    const int plane_u = sm.plane_u, plane_a = sm.plane_a;
    const float *ring = sm.ring;
    const float *aux = sm.aux;
    volatile int *abort_flag = sm.abort;
    auto BAR = [&](int i) { return smem_addr(&sm.bars[i]); };

    const bool active = r < rows && col0 + 4 * qc < a.n2;
    constexpr bool kImgRegs = IMG && M <= 6;
    float4 img_cur[4], img_next[4];
#pragma unroll
    for (int k = 0; k < 4; k++) img_cur[k] = img_next[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    auto img_fetch = [&](int zo_f, float4 (&dst)[4]) {
        const long long at = (long long)zo_f * a.s0 + (long long)(row0 + r) * a.s1 + col0 + 4 * qc;
        const float *src[4] = {img.u0, img.u1, img.u2, img.grad};
        if (col0 + 4 * qc + 3 < a.n2) {
#pragma unroll
            for (int k = 0; k < 4; k++) dst[k] = *reinterpret_cast<const float4 *>(src[k] + at);
        } else {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (col0 + 4 * qc + i < a.n2) v[i] = src[k][at + i];
                dst[k] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    };
    auto img_prefetch_l2 = [&](int zo_f) {
        const long long at = (long long)zo_f * a.s0 + (long long)(row0 + r) * a.s1 + col0 + 4 * qc;
        const float *src[4] = {img.u0, img.u1, img.u2, img.grad};
#pragma unroll
        for (int k = 0; k < 4; k++) asm volatile("prefetch.global.L2 [%0];" ::"l"(src[k] + at));
    };

    constexpr int Q = 2 * M + 1;  // d0 queue length
    float4 q[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    bool ok = true;
#pragma unroll(M >= 6 ? 2 : 1)
    for (int j = 0; j < J; j++) {
        if constexpr (IMG) {
            const int zn = z_lo + j + 1 - 2 * M;
            if (active && zn + 2 >= z_lo && zn + 2 < z_hi) img_prefetch_l2(zn + 2);
            if (kImgRegs && active && zn >= z_lo && zn < z_hi) img_fetch(zn, img_next);
        }
        const unsigned U = ub + (unsigned)j;
        ok = mbar_wait_flag(BAR((int)(U % NU)), (U / NU) & 1, abort_flag);
#pragma unroll
        for (int k = 0; k < Q - 1; k++) q[k] = q[k + 1];
        q[Q - 1] = *reinterpret_cast<const float4 *>(ring + (U % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc);
        if (ok && j >= 2 * M) {
            const int ja = j - 2 * M;  // output plane z_lo + ja
            const int zo = z_lo + ja;
            const unsigned A = ab + (unsigned)ja;
            ok = mbar_wait_flag(BAR(kFullA + (int)(A % NA)), (A / NA) & 1, abort_flag);
            if (ok && active) {
                if constexpr (IMG && !kImgRegs) img_fetch(zo, img_cur);
                update_points<M, IMG>(ring + ((U - M) % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc,
                                      aux + (A % NA) * 3 * plane_a + r * kTileW + 4 * qc, plane_a, q, cf, a,
                                      row0, col0, r, qc, zo, out, nsrc, sm.src, sm.sstart, src_row, img, img_cur);
            }
        }
        if constexpr (kImgRegs) {
#pragma unroll
            for (int k = 0; k < 4; k++) img_cur[k] = img_next[k];
        }
        if (!ok) break;
        // Every thread fences its shared-memory reads (generic proxy) against
        // the TMA copies (async proxy) that will refill the slots, then
        // hands them back: without the fence a refill could overtake reads
        // still in flight (measured: results that differed from run to run
        // whenever another kernel shared the SMs).
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (j < M || j >= J - M) mbar_arrive_cta(BAR(kEmptyU + (int)(U % NU)));
        if (j >= 2 * M) {
            mbar_arrive_cta(BAR(kEmptyU + (int)((U - M) % NU)));
            mbar_arrive_cta(BAR(kEmptyA + (int)((ab + (unsigned)(j - 2 * M)) % NA)));
        }
        if (*abort_flag) {
            ok = false;
            break;
        }
    }
    if (!ok && lane == 0) {
        *abort_flag = 1;
        atomicCAS(status, 0, (int)FD_ERR_TIMEOUT);
    }
    return ok;
}

// One tile column per CTA (the single-grid kernel): stage the column's
// corners (every thread), then the last warp produces and the others
// compute.
template <int M, int P, bool IMG = false>
__device__ void sweep_column_ws(const CUtensorMap *map_u, const CUtensorMap *map_um, const CUtensorMap *map_c,
                                const CUtensorMap *map_d, float *__restrict__ out, const TileArgs &a, const Coef &cf,
                                int tile, int z_lo, int z_hi, const SrcEntry *__restrict__ src_tab, int nsrc,
                                const float *__restrict__ src_row, const SweepSmem &sm, int *status,
                                const ImagingArgs &img = ImagingArgs())
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int compute_warps = (int)(blockDim.x >> 5) - 1;
    if (!src_row) nsrc = 0;
    stage_sources(src_tab, nsrc, a.n0, sm, (int)blockDim.x, [] { __syncthreads(); });
    if (warp == compute_warps) {
        if (lane == 0) {
            unsigned nu = 0, na = 0;
            if (!ws_produce_column<M, P>(map_u, map_um, map_c, map_d, a, tile, z_lo, z_hi, sm, nu, na))
                ws_drain<M, P>(sm, nu, na, status);
        }
        __syncwarp();
        return;
    }
    ws_consume_column<M, P, IMG>(a, cf, tile, z_lo, z_hi, out, nsrc, src_row, sm, 0u, 0u, status, img);
}

}  // namespace tile_dev

}  // namespace fdgb
