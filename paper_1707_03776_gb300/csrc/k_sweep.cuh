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
// One elected thread issues the copies P planes ahead on mbarriers with
// transaction counts; every wait is bounded by the global timer and, when it
// gives up, the CTA records FD_ERR_TIMEOUT in the status word and leaves after
// draining its own copies.
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
// ring, the aux ring, the mbarriers, the abort flag and the batch kernel's
// item slot (16 bytes), then src_cap
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
    l.abort = l.bars + sizeof(unsigned long long) * (size_t)(2 * (NU + NA));  // full and empty
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
    unsigned long long *bars;    // NU + NA mbarriers
    volatile int *abort;
    int *item;                   // batch kernel: the work item being taken (next to abort)
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
    sm.item = reinterpret_cast<int *>(raw + l.abort) + 1;
    sm.src = reinterpret_cast<SrcEntry *>(raw + l.src);
    sm.sstart = reinterpret_cast<int *>(raw + l.sstart);
    return sm;
}

template <int M, int P>
__device__ inline void init_barriers(const SweepSmem &sm)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < M + 1 + P + P + 1; i++) mbar_init(smem_addr(&sm.bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *sm.abort = 0;
    }
    __syncthreads();
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

// Sweep output planes [z_lo, z_hi) of tile `tile` of one grid (the first 2M
// iterations only load the u^n planes z_lo-M .. z_lo+M-1 that the first
// output plane reads).  it_u / it_a count the u^n and aux loads this CTA has
// consumed so far (ring slots and barrier phases continue across columns).
// Returns false when a wait gave up (status set, copies drained).
// With IMG, the imaging condition of `img` is accumulated at every point
// written, from the value written (sources included).
template <int M, int P, bool IMG = false>
__device__ bool sweep_column(const CUtensorMap *map_u, const CUtensorMap *map_um, const CUtensorMap *map_c,
                             const CUtensorMap *map_d, float *__restrict__ out, const TileArgs &a, const Coef &cf,
                             int tile, int z_lo, int z_hi, const SrcEntry *__restrict__ src_tab, int nsrc,
                             const float *__restrict__ src_row, const SweepSmem &sm, unsigned &it_u, unsigned &it_a,
                             int *status, const ImagingArgs &img = ImagingArgs())
{
    constexpr int NU = M + 1 + P;     // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;         // aux planes (u^{n-1}, c, d)
    constexpr int HV = (M + 3) / 4;   // float4 groups on each side of a thread's 4 points
    constexpr int NR = 4 * (2 * HV + 1);
    constexpr int Q = 2 * M + 1;      // d0 queue length

    const int tid = threadIdx.x;
    const int strip = tile / a.k2;
    const int tile2 = tile - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = tile2 * kTileW;
    const int r = tid >> 4;
    const int qc = tid & 15;
    const bool active = r < rows && col0 + 4 * qc < a.n2;
    const int J = (z_hi - z_lo) + 2 * M;
    const int plane_u = sm.plane_u, plane_a = sm.plane_a;
    float *ring = sm.ring;
    float *aux = sm.aux;
    unsigned long long *bars = sm.bars;
    const uint32_t bytes_u = (uint32_t)(kBoxW * a.box_h * sizeof(float));
    const uint32_t bytes_a = (uint32_t)(3 * a.rows_max * kTileW * sizeof(float));
    const unsigned iu = it_u, ia = it_a;

    // iteration j: u^n plane z_lo-M+j into ring slot (iu+j) % NU; for j >= 2M
    // the aux of output plane z_lo+j-2M into aux slot (ia+j-2M) % NA
    auto issue = [&](int j) {
        const unsigned gu = iu + (unsigned)j;
        const int su = (int)(gu % NU);
        const uint32_t bu = smem_addr(&bars[su]);
        mbar_expect_tx(bu, bytes_u);
        // the stall hook arms the barrier but never issues the copy, so the
        // wait for this plane runs out (the failure path under test)
        if (a.stall_plane < 0 || tile != 0 || z_lo - M + j != a.stall_plane)
            tma_load_3d(smem_addr(ring + su * plane_u), map_u, col0 - kSideHalo, row0 - M, z_lo - M + j, bu);
        if (j >= 2 * M) {
            const int ja = j - 2 * M;
            const int sa = (int)((ia + (unsigned)ja) % NA);
            const uint32_t ba = smem_addr(&bars[NU + sa]);
            float *dst = aux + sa * 3 * plane_a;
            mbar_expect_tx(ba, bytes_a);
            tma_load_3d(smem_addr(dst), map_um, col0, row0, z_lo + ja, ba);
            tma_load_3d(smem_addr(dst + plane_a), map_c, col0, row0, z_lo + ja, ba);
            tma_load_3d(smem_addr(dst + 2 * plane_a), map_d, col0, row0, z_lo + ja, ba);
        }
    };
    auto wait_u = [&](int j) {
        const unsigned gu = iu + (unsigned)j;
        return mbar_wait_bounded(smem_addr(&bars[gu % NU]), (uint32_t)((gu / NU) & 1));
    };
    auto wait_a = [&](int ja) {
        const unsigned ga = ia + (unsigned)ja;
        return mbar_wait_bounded(smem_addr(&bars[NU + ga % NA]), (uint32_t)((ga / NA) & 1));
    };

    if (tid == 0)
        for (int j = 0; j < P && j < J; j++) issue(j);

    // the column's injected corners, staged in shared memory so that the
    // plane loop never waits on them
    SrcEntry *s_src = sm.src;
    int *s_sstart = sm.sstart;
    if (!src_row) nsrc = 0;
    for (int q = tid; q < nsrc * 5; q += blockDim.x)
        reinterpret_cast<int *>(s_src)[q] = reinterpret_cast<const int *>(src_tab)[q];
    __syncthreads();
    if (nsrc > 0) {
        for (int z = tid; z <= a.n0; z += blockDim.x) {
            int lo = 0, hi = nsrc;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_src[mid].z < z) lo = mid + 1; else hi = mid;
            }
            s_sstart[z] = lo;
        }
        __syncthreads();
    }

    // d0 queue: q[k] holds the thread's 4 centre values of plane z - M + k
    // for the output plane z of the current iteration (shifted each plane)
    float4 q[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);

    // imaging inputs (u0, u1, u2, grad) of the next output plane, loaded one
    // iteration ahead into registers (up to M = 6; the highest orders load
    // them when used), after an L2 prefetch three iterations ahead, so that
    // their DRAM latency overlaps planes of work
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

    int j = 0;
    bool ok = true, stop = false;
    // at high orders the d0 queue shift (2M+1 float4 moves per plane) is a
    // large share of the instructions: unrolling two planes lets them be
    // renamed instead (measured: SO12/16 about 5 % faster, SO8 1.4 % slower)
#pragma unroll(M >= 6 ? 2 : 1)
    for (; j < J; j++) {
        if (tid == 0 && j + P < J) issue(j + P);
        if constexpr (IMG) {
            // output plane of the next iteration into registers, and the one
            // two further into L2 (so that the register loads find it there)
            const int zn = z_lo + j + 1 - 2 * M;
            if (active && zn + 2 >= z_lo && zn + 2 < z_hi) img_prefetch_l2(zn + 2);
            if (kImgRegs && active && zn >= z_lo && zn < z_hi) img_fetch(zn, img_next);
        }
        ok = wait_u(j) && ok;
#pragma unroll
        for (int k = 0; k < Q - 1; k++) q[k] = q[k + 1];
        q[Q - 1] = *reinterpret_cast<const float4 *>(ring + ((iu + j) % NU) * plane_u + (r + M) * kBoxW + kSideHalo +
                                                     4 * qc);
        if (j >= 2 * M) {
            const int ja = j - 2 * M;  // output plane z_lo + ja
            const int zo = z_lo + ja;
            ok = wait_a(ja) && ok;
            if (ok && active) {
                if constexpr (IMG && !kImgRegs) img_fetch(zo, img_cur);
                update_points<M, IMG>(ring + ((iu + j - M) % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc,
                                      aux + ((ia + ja) % NA) * 3 * plane_a + r * kTileW + 4 * qc, plane_a, q, cf, a,
                                      row0, col0, r, qc, zo, out, nsrc, s_src, s_sstart, src_row, img, img_cur);
            }
        }
        if constexpr (kImgRegs) {
#pragma unroll
            for (int k = 0; k < 4; k++) img_cur[k] = img_next[k];
        }
        if (!ok) *sm.abort = 1;
        // the ring slots read above are refilled by TMA (async proxy) after
        // this barrier: fence the generic-proxy reads against that
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (*sm.abort) {
            stop = true;
            break;
        }
    }

    if (stop) {
        // a wait gave up: record it, then drain this CTA's copies still in
        // flight (issued up to min(j+P, J-1)) before leaving.  Every barrier
        // is waited on, under one shared deadline, so that a copy that never
        // lands does not stop the drain short of the ones behind it.
        if (tid == 0) {
            atomicExch(status, (int)FD_ERR_TIMEOUT);
            const unsigned long long deadline = global_ns() + kWaitLimitNs;
            const int last = (j + P < J) ? j + P : J - 1;
            for (int i = j; i <= last; i++) {
                const unsigned gu = iu + (unsigned)i;
                mbar_wait_until(smem_addr(&bars[gu % NU]), (uint32_t)((gu / NU) & 1), deadline);
                if (i >= 2 * M) {
                    const unsigned ga = ia + (unsigned)(i - 2 * M);
                    mbar_wait_until(smem_addr(&bars[NU + ga % NA]), (uint32_t)((ga / NA) & 1), deadline);
                }
            }
        }
        __syncthreads();
        return false;
    }
    it_u = iu + (unsigned)J;
    it_a = ia + (unsigned)(z_hi - z_lo);
    return true;
}

// The sweep of one tile column with a producer warp (the single-grid tiled
// kernel): the CTA's last warp issues the copies, P planes ahead, into ring
// slots that the compute warps hand back through "empty" mbarriers (one
// arrival per compute thread after its last read of the slot), so that a
// compute warp waits only for its own data, never for the other warps, and
// warps may drift up to P planes apart.  Same arithmetic as sweep_column
// (update_points).  Barriers: full u^n [NU], full aux [NA], empty u^n [NU],
// empty aux [NA]; every wait is bounded, a wait that gives up records
// FD_ERR_TIMEOUT and raises the CTA's abort flag, which every role checks;
// the producer then drains the copies it still owes.  One column per CTA:
// slots are not reused across columns.
template <int M, int P>
__device__ inline void init_barriers_ws(const SweepSmem &sm, unsigned compute_warps)
{
    constexpr int NU = M + 1 + P, NA = P + 1;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NU + NA; i++) mbar_init(smem_addr(&sm.bars[i]), 1);
        for (int i = NU + NA; i < 2 * (NU + NA); i++) mbar_init(smem_addr(&sm.bars[i]), 32 * compute_warps);
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

template <int M, int P, bool IMG = false>
__device__ void sweep_column_ws(const CUtensorMap *map_u, const CUtensorMap *map_um, const CUtensorMap *map_c,
                                const CUtensorMap *map_d, float *__restrict__ out, const TileArgs &a, const Coef &cf,
                                int tile, int z_lo, int z_hi, const SrcEntry *__restrict__ src_tab, int nsrc,
                                const float *__restrict__ src_row, const SweepSmem &sm, int *status,
                                const ImagingArgs &img = ImagingArgs())
{
    constexpr int NU = M + 1 + P;     // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;         // aux planes (u^{n-1}, c, d)
    constexpr int Q = 2 * M + 1;      // d0 queue length
    constexpr int kFullA = NU, kEmptyU = NU + NA, kEmptyA = 2 * NU + NA;

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int compute_warps = (int)(blockDim.x >> 5) - 1;
    const int strip = tile / a.k2;
    const int tile2 = tile - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = tile2 * kTileW;
    const int r = tid >> 4;
    const int qc = tid & 15;
    const int J = (z_hi - z_lo) + 2 * M;
    const int plane_u = sm.plane_u, plane_a = sm.plane_a;
    float *ring = sm.ring;
    float *aux = sm.aux;
    unsigned long long *bars = sm.bars;
    volatile int *abort_flag = sm.abort;
    auto BAR = [&](int i) { return smem_addr(&bars[i]); };

    // the column's injected corners, staged in shared memory (all threads)
    SrcEntry *s_src = sm.src;
    int *s_sstart = sm.sstart;
    if (!src_row) nsrc = 0;
    for (int q = tid; q < nsrc * 5; q += blockDim.x)
        reinterpret_cast<int *>(s_src)[q] = reinterpret_cast<const int *>(src_tab)[q];
    __syncthreads();
    if (nsrc > 0) {
        for (int z = tid; z <= a.n0; z += blockDim.x) {
            int lo = 0, hi = nsrc;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_src[mid].z < z) lo = mid + 1; else hi = mid;
            }
            s_sstart[z] = lo;
        }
        __syncthreads();
    }

    if (warp == compute_warps) {
        // producer: sweep plane j of u^n into slot j % NU; for j >= 2M the
        // aux of output plane j - 2M into slot (j - 2M) % NA
        if (lane == 0) {
            const uint32_t bytes_u = (uint32_t)(kBoxW * a.box_h * sizeof(float));
            const uint32_t bytes_a = (uint32_t)(3 * a.rows_max * kTileW * sizeof(float));
            int ju = 0, jaux = 0;  // u planes / aux planes issued
            bool ok = true;
            for (int j = 0; j < J && ok; j++) {
                const int su = j % NU;
                // the slot's previous plane j - NU was last read at iteration
                // j - NU + M (as the centre plane) or j - NU (if j - NU < M)
                if (j >= NU && !mbar_wait_flag(BAR(kEmptyU + su), (uint32_t)(((j / NU) - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(BAR(su), bytes_u);
                // the stall hook arms the barrier but never issues the copy,
                // so the wait for this plane runs out (the failure path under test)
                if (a.stall_plane < 0 || tile != 0 || z_lo - M + j != a.stall_plane)
                    tma_load_3d(smem_addr(ring + su * plane_u), map_u, col0 - kSideHalo, row0 - M, z_lo - M + j,
                                BAR(su));
                ju++;
                if (j >= 2 * M) {
                    const int ja = j - 2 * M;
                    const int sa = ja % NA;
                    if (ja >= NA && !mbar_wait_flag(BAR(kEmptyA + sa), (uint32_t)(((ja / NA) - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    float *dst = aux + sa * 3 * plane_a;
                    mbar_expect_tx(BAR(kFullA + sa), bytes_a);
                    tma_load_3d(smem_addr(dst), map_um, col0, row0, z_lo + ja, BAR(kFullA + sa));
                    tma_load_3d(smem_addr(dst + plane_a), map_c, col0, row0, z_lo + ja, BAR(kFullA + sa));
                    tma_load_3d(smem_addr(dst + 2 * plane_a), map_d, col0, row0, z_lo + ja, BAR(kFullA + sa));
                    jaux++;
                }
            }
            if (!ok || *abort_flag) {
                // drain the copies possibly still in flight (the last of each
                // ring), under one shared deadline
                *abort_flag = 1;
                atomicExch(status, (int)FD_ERR_TIMEOUT);
                const unsigned long long deadline = global_ns() + kWaitLimitNs;
                for (int k = ju > NU ? ju - NU : 0; k < ju; k++)
                    mbar_wait_until(BAR(k % NU), (uint32_t)((k / NU) & 1), deadline);
                for (int k = jaux > NA ? jaux - NA : 0; k < jaux; k++)
                    mbar_wait_until(BAR(kFullA + k % NA), (uint32_t)((k / NA) & 1), deadline);
            }
        }
        __syncwarp();
        return;
    }

    // compute warps
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
        ok = mbar_wait_flag(BAR(j % NU), (uint32_t)((j / NU) & 1), abort_flag);
#pragma unroll
        for (int k = 0; k < Q - 1; k++) q[k] = q[k + 1];
        q[Q - 1] = *reinterpret_cast<const float4 *>(ring + (j % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc);
        if (ok && j >= 2 * M) {
            const int ja = j - 2 * M;  // output plane z_lo + ja
            const int zo = z_lo + ja;
            ok = mbar_wait_flag(BAR(kFullA + ja % NA), (uint32_t)((ja / NA) & 1), abort_flag);
            if (ok && active) {
                if constexpr (IMG && !kImgRegs) img_fetch(zo, img_cur);
                update_points<M, IMG>(ring + ((j - M) % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc,
                                      aux + (ja % NA) * 3 * plane_a + r * kTileW + 4 * qc, plane_a, q, cf, a,
                                      row0, col0, r, qc, zo, out, nsrc, s_src, s_sstart, src_row, img, img_cur);
            }
        }
        if constexpr (kImgRegs) {
#pragma unroll
            for (int k = 0; k < 4; k++) img_cur[k] = img_next[k];
        }
        if (!ok) break;
        // hand back the slots read for the last time: u^n plane j - M (the
        // centre just used) -- or plane j itself while j < M -- and the aux
        // of output plane j - 2M.  Every thread fences its shared-memory
        // reads (generic proxy) against the TMA copies (async proxy) that will
        // refill the slots, then arrives: without the fence the refill could
        // overtake reads still in flight (measured: results that differed
        // from run to run whenever another kernel shared the SMs).
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (j < M) mbar_arrive_cta(BAR(kEmptyU + j % NU));
        else if (j >= 2 * M) mbar_arrive_cta(BAR(kEmptyU + (j - M) % NU));
        if (j >= 2 * M) mbar_arrive_cta(BAR(kEmptyA + (j - 2 * M) % NA));
        if (*abort_flag) break;
    }
    if (!ok && lane == 0) {
        *abort_flag = 1;
        atomicExch(status, (int)FD_ERR_TIMEOUT);
    }
}

}  // namespace tile_dev

}  // namespace fdgb
