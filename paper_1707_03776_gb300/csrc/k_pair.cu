// Temporal blocking of the 3D acoustic grid update: two time steps of the
// leapfrog update (Section "Acoustic wave equation", the solved stencil for
// u^{n+1}) in one sweep over the grid.
//
// One cooperative launch, one CTA per tile column (64 columns of d2, a strip
// of d1 rows, every d0 plane), every column resident at once.  Each CTA
// streams its column along d0 with two stages, the second L = max(M, 4)
// planes behind the first:
//   stage 1  u^{n+1} at plane p from u^n (haloed TMA ring + the d0 register
//            queue q0), u^{n-1}, c and d: the single-step sweep.  The result
//            is written in place over u^{n-1} and pushed into a second
//            register queue q1;
//   stage 2  u^{n+2} at plane p - L: the d1/d2 neighbours from a haloed TMA
//            box of u^{n+1} (its halo rows and columns were written by the
//            neighbouring columns' stage 1 a few planes earlier and are still
//            in L2), the d0 neighbours from q1, u^n from the oldest entry of
//            q0, c and d from a second TMA load (also L2).  The result is
//            written in place over u^n.
// Per point and two steps HBM sees u^n, u^{n-1}, c and d read once and the
// two new fields written once: 24 bytes instead of the 40 of two sweeps.
// Both stages evaluate the same expression in the same order as the
// single-step kernel, so the two are bitwise equal.
//
// Ordering between columns.  A haloed box reaches only the adjacent columns
// (strips are at least M rows tall, interior tiles 64 >= 8 columns wide).
// After stage 1 has stored plane p, thread 0 publishes the column's progress
// (planes of u^{n+1} written) with a release store.  The stage-2 box of plane
// q is loaded once the (up to 8) neighbouring columns have published q + 1:
// warp 0 reads the eight flags with eight lanes at once (acquire, bounded by
// the global timer) and keeps the smallest value seen, so that most
// iterations read none.  That one condition also makes the in-place write of
// u^{n+2} safe: a neighbour that has finished stage 1 at plane q has loaded
// every u^n plane up to q + M.  Stage 1 reads only the launch's inputs and
// never waits, and at iteration j a column waits only on columns that have
// reached iteration j - L + 2 (two planes of slack in lockstep), so no wait
// closes a cycle.  A wait that gives up records FD_ERR_TIMEOUT, every other
// column's wait gives up as soon as it sees a non-zero status, and each CTA
// drains the copies it issued before it returns.
//
// Measured on the 512^3 SO8 workload the sweep is slower than two single-step
// sweeps: a gpu-scope release under full HBM load takes 3-6 us, several
// plane-iterations, so the columns wait on one another's flags; hiding it
// would take a lag of 6-8 planes, which the registers (two queues) and the
// shared memory (two pipelines) of one CTA per SM do not hold.  The operator
// therefore steps one at a time unless two steps per sweep are asked for.
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "fd_internal.h"
#include "fd_internal_host.h"
#include "k_sweep.cuh"

namespace fdgb {

namespace {

using namespace tile_dev;

constexpr int kPairThreads = 448;                // 28 rows of 16 threads
constexpr int kPairMaxRows = kPairThreads / 16;
constexpr int kPairStages = 2;                   // u^n planes in flight

// Byte offsets of a two-step CTA's dynamic shared memory: the u^n ring
// (M + 1 + P haloed planes), two haloed u^{n+1} boxes, P + 1 slots of
// (u^{n-1}, c, d) tiles for stage 1, two slots of (c, d) tiles for stage 2,
// the mbarriers, the abort flag (16 bytes), then src_cap injected corners and
// their n0 + 1 per-plane starts.
struct PairLayout {
    size_t box, aux1, aux2, bars, abort, src, sstart, end;
};

__host__ __device__ inline int pair_barriers(int M, int P) { return (M + 1 + P) + (P + 1) + 2; }

__host__ __device__ inline PairLayout pair_smem_layout(int M, int P, int rows_max, int src_cap, int n0)
{
    const size_t plane = sizeof(float) * (size_t)ring_plane_floats(rows_max + 2 * M);
    const size_t tile = sizeof(float) * (size_t)rows_max * kTileW;
    PairLayout l;
    l.box = (size_t)(M + 1 + P) * plane;
    l.aux1 = l.box + 2 * plane;
    l.aux2 = l.aux1 + (size_t)(P + 1) * 3 * tile;
    l.bars = l.aux2 + 2 * 2 * tile;
    l.abort = l.bars + sizeof(unsigned long long) * (size_t)pair_barriers(M, P);
    l.src = l.abort + 16;
    l.sstart = l.src + sizeof(SrcEntry) * (size_t)src_cap;
    l.end = l.sstart + sizeof(int) * (size_t)(n0 + 1);
    return l;
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// orders this thread's generic-proxy global accesses with later TMA
// (async-proxy) accesses
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The update at a thread's 4 consecutive d2 points: pc points at the first of
// them in a haloed plane (row stride kBoxW), q[OFF .. OFF+2M] holds the 2M+1
// values along d0 (centre q[OFF+M]); umv, cv, dv are u^{n-1}, c and d there.
template <int M, int OFF, int QN>
__device__ __forceinline__ void update4(const float *pc, const float4 (&q)[QN], const float umv[4],
                                        const float cv[4], const float dv[4], const Coef &cf, float res[4])
{
    static_assert(OFF + 2 * M < QN, "queue window");
    constexpr int HV = (M + 3) / 4;  // float4 groups on each side of the thread's 4 points
    constexpr int NR = 4 * (2 * HV + 1);
    float row[NR];
#pragma unroll
    for (int v = 0; v < 2 * HV + 1; v++) {
        const float4 t = *reinterpret_cast<const float4 *>(pc + 4 * (v - HV));
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
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float u = row[4 * HV + i];
        float lap = cf.centre * u;
#pragma unroll
        for (int k = 1; k <= M; k++) {
            const float4 lo = q[OFF + M - k];
            const float4 hi = q[OFF + M + k];
            const float s2 = row[4 * HV + i - k] + row[4 * HV + i + k];
            const float s1 = (&cm[k].x)[i] + (&cp[k].x)[i];
            const float s0 = (&lo.x)[i] + (&hi.x)[i];
            lap = fmaf(cf.ax[2][k], s2, lap);
            lap = fmaf(cf.ax[1][k], s1, lap);
            lap = fmaf(cf.ax[0][k], s0, lap);
        }
        // the tiled kernel's chain of three FMAs
        res[i] = fmaf(-dv[i], u - umv[i], fmaf(cv[i], lap, fmaf(2.0f, u, -umv[i])));
    }
}

// Source injection at the corners of plane z that the thread (row r, float4
// column qc) owns: res += c * w * src_row[p].
__device__ __forceinline__ void inject4(float res[4], const float cv[4], const SrcEntry *s_src, const int *s_sstart,
                                        int z, int r, int qc, const float *src_row)
{
    float inj0 = 0.f, inj1 = 0.f, inj2 = 0.f, inj3 = 0.f;
    const int s_end = s_sstart[z + 1];
    for (int k = s_sstart[z]; k < s_end; k++) {
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

__device__ __forceinline__ void store4(float *out, const TileArgs &a, int z, int row, int col, const float res[4])
{
    float *o = out + (long long)z * a.s0 + (long long)row * a.s1 + col;
    if (col + 3 < a.n2) {
        *reinterpret_cast<float4 *>(o) = make_float4(res[0], res[1], res[2], res[3]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (col + i < a.n2) o[i] = res[i];
    }
}

// map_u0: u^n, haloed box; map_um: u^{n-1}, tile box; map_c / map_d: tile
// boxes; map_u1: u^{n+1} (the buffer of u^{n-1}), haloed box.  out1 is the
// buffer of u^{n-1} (receives u^{n+1}), out2 that of u^n (receives u^{n+2}).
template <int M, int P>
__global__ void __launch_bounds__(kPairThreads, 1)
    acoustic_pair_kernel(const __grid_constant__ CUtensorMap map_u0, const __grid_constant__ CUtensorMap map_um,
                         const __grid_constant__ CUtensorMap map_c, const __grid_constant__ CUtensorMap map_d,
                         const __grid_constant__ CUtensorMap map_u1, float *out1, float *out2, const TileArgs a,
                         const Coef cf, int *status, int *progress, const SrcEntry *__restrict__ src_tab,
                         const int *__restrict__ src_off, const float *src_row1, const float *src_row2,
                         const int src_cap)
{
    constexpr int NU = M + 1 + P;  // u^n planes alive: M behind the newest, the newest, P in flight
    constexpr int NA = P + 1;      // stage-1 (u^{n-1}, c, d) slots
    constexpr int L = M > 4 ? M : 4;  // stage 2 trails stage 1 by L planes
    constexpr int E = L - M;
    constexpr int Q = 2 * M + 1 + E;  // d0 queues: the stencil window plus E planes of lag
    static_assert(M >= 2 && L >= M, "two planes of slack need L >= M >= 2");

    if (*reinterpret_cast<volatile int *>(status) != 0) return;
    const PairLayout lay = pair_smem_layout(M, P, a.rows_max, src_cap, a.n0);
    if (lay.end > (size_t)dynamic_smem_bytes()) {
        if (threadIdx.x == 0) atomicExch(status, (int)FD_ERR_LAYOUT);
        return;
    }
    const int tile = (int)blockIdx.x;
    const bool with_src = src_row1 != nullptr && src_row2 != nullptr;
    const int s0 = with_src ? src_off[tile] : 0;
    const int nsrc = with_src ? src_off[tile + 1] - s0 : 0;
    if (nsrc > src_cap) {
        if (threadIdx.x == 0) atomicExch(status, (int)FD_ERR_LAYOUT);
        return;
    }

    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *ring = reinterpret_cast<float *>(smem_raw);
    float *box = reinterpret_cast<float *>(smem_raw + lay.box);
    float *aux1 = reinterpret_cast<float *>(smem_raw + lay.aux1);
    float *aux2 = reinterpret_cast<float *>(smem_raw + lay.aux2);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_raw + lay.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem_raw + lay.abort);
    SrcEntry *s_src = reinterpret_cast<SrcEntry *>(smem_raw + lay.src);
    int *s_sstart = reinterpret_cast<int *>(smem_raw + lay.sstart);

    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_map(&map_u0);
        prefetch_map(&map_um);
        prefetch_map(&map_c);
        prefetch_map(&map_d);
        prefetch_map(&map_u1);
        for (int i = 0; i < pair_barriers(M, P); i++) mbar_init(smem_addr(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    __syncthreads();

    const int strip = tile / a.k2;
    const int t2 = tile - strip * a.k2;
    const int row0 = (int)((long long)strip * a.n1 / a.k1);
    const int rows = (int)((long long)(strip + 1) * a.n1 / a.k1) - row0;
    const int col0 = t2 * kTileW;
    const int r = tid >> 4;
    const int qc = tid & 15;
    const bool active = r < rows && col0 + 4 * qc < a.n2;
    const int plane_u = ring_plane_floats(a.box_h);
    const int plane_a = a.rows_max * kTileW;
    const int J1 = a.n0 + 2 * M;  // iterations that load u^n; stage 1 finishes plane j - 2M
    const int J = a.n0 + 2 * M + L;  // stage 2 finishes plane j - 2M - L
    const uint32_t bytes_u = (uint32_t)(kBoxW * a.box_h * sizeof(float));
    const uint32_t bytes_a1 = (uint32_t)(3 * plane_a * sizeof(float));
    const uint32_t bytes_2 = bytes_u + (uint32_t)(2 * plane_a * sizeof(float));

    auto bar = [&](int i) { return smem_addr(&bars[i]); };
    // iteration j: u^n plane j - M into ring slot j % NU; for j >= 2M the
    // (u^{n-1}, c, d) tiles of plane j - 2M into slot (j - 2M) % NA
    auto issue1 = [&](int j) {
        const int su = j % NU;
        mbar_expect_tx(bar(su), bytes_u);
        // the stall hook arms the barrier but never issues the copy, so the
        // wait for this plane runs out (the failure path under test)
        if (a.stall_plane < 0 || tile != 0 || j - M != a.stall_plane)
            tma_load_3d(smem_addr(ring + su * plane_u), &map_u0, col0 - kSideHalo, row0 - M, j - M, bar(su));
        if (j >= 2 * M) {
            const int ja = j - 2 * M;
            const int sa = ja % NA;
            float *dst = aux1 + sa * 3 * plane_a;
            mbar_expect_tx(bar(NU + sa), bytes_a1);
            tma_load_3d(smem_addr(dst), &map_um, col0, row0, ja, bar(NU + sa));
            tma_load_3d(smem_addr(dst + plane_a), &map_c, col0, row0, ja, bar(NU + sa));
            tma_load_3d(smem_addr(dst + 2 * plane_a), &map_d, col0, row0, ja, bar(NU + sa));
        }
    };
    // iteration j >= 2M + L: the haloed u^{n+1} box and the c, d tiles of
    // plane j - 2M - L into slot (j - 2M - L) & 1
    auto issue2 = [&](int j) {
        const int jb = j - 2 * M - L;
        const int sb = jb & 1;
        const uint32_t b2 = bar(NU + NA + sb);
        mbar_expect_tx(b2, bytes_2);
        tma_load_3d(smem_addr(box + sb * plane_u), &map_u1, col0 - kSideHalo, row0 - M, jb, b2);
        float *dst = aux2 + sb * 2 * plane_a;
        tma_load_3d(smem_addr(dst), &map_c, col0, row0, jb, b2);
        tma_load_3d(smem_addr(dst + plane_a), &map_d, col0, row0, jb, b2);
    };
    auto wait_u = [&](int j) { return mbar_wait_bounded(bar(j % NU), (uint32_t)((j / NU) & 1)); };
    auto wait_a = [&](int ja) { return mbar_wait_bounded(bar(NU + ja % NA), (uint32_t)((ja / NA) & 1)); };
    auto wait_b = [&](int jb) { return mbar_wait_bounded(bar(NU + NA + (jb & 1)), (uint32_t)((jb >> 1) & 1)); };
    // warp 0: until every neighbouring column has written u^{n+1} planes
    // [0, need).  Lane l < 8 reads the flag of neighbour l; seen keeps the
    // smallest value read, so a wait already covered reads nothing.  Gives up
    // after the wait limit, or at once when a CTA has recorded an error.
    const int *nb_flag = nullptr;
    if (tid < 8) {
        const int o = tid < 4 ? tid : tid + 1;  // 3 x 3 neighbourhood without its centre
        const int s = strip + o / 3 - 1, t = t2 + o % 3 - 1;
        if (s >= 0 && s < a.k1 && t >= 0 && t < a.k2) nb_flag = progress + s * a.k2 + t;
    }
    int seen = -1;
    auto neighbours_ready = [&](int need) {
        if (seen >= need) return true;
        const unsigned long long t0 = global_ns();
        for (;;) {
            const int v = nb_flag ? ld_acquire(nb_flag) : 0x7fffffff;
            seen = __reduce_min_sync(0xffffffffu, v);
            if (seen >= need) break;
            const bool give_up =
                *reinterpret_cast<volatile int *>(status) != 0 || global_ns() - t0 > kWaitLimitNs;
            if (__any_sync(0xffffffffu, give_up)) return false;
        }
        __syncwarp();
        return true;
    };

    int issued1 = -1, issued2 = -1;  // last iterations whose copies thread 0 issued
    if (tid == 0)
        for (int j = 0; j < P && j < J1; j++) {
            issue1(j);
            issued1 = j;
        }

    // the column's injected corners, staged in shared memory
    for (int q = tid; q < nsrc * 5; q += blockDim.x)
        reinterpret_cast<int *>(s_src)[q] = reinterpret_cast<const int *>(src_tab + s0)[q];
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

    // after the pushes of iteration j: q0[k] holds u^n at plane
    // j - 3M - E + k (the thread's 4 points), q1[k] u^{n+1} at plane
    // j - 3M - L + k
    float4 q0[Q], q1[Q];
#pragma unroll
    for (int k = 0; k < Q; k++) {
        q0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        q1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    int j = 0;
    bool ok = true, stop = false;
    for (; j < J; j++) {
        if (tid < 32) {
            if (tid == 0 && j + P < J1) {
                issue1(j + P);
                issued1 = j + P;
            }
            const int jn = j + 1;
            if (jn >= 2 * M + L && jn < J) {
                // this column has written planes [0, j - 2M), >= jn - 2M - L + 2
                if (neighbours_ready(jn - 2 * M - L + 1)) {
                    if (tid == 0) {
                        fence_proxy_async_global();
                        issue2(jn);
                        issued2 = jn;
                    }
                } else if (tid == 0) {
                    *abort_flag = 1;
                }
            }
        }

        // stage 1: the newest u^n plane (j - M) into q0, u^{n+1} at j - 2M
        if (j < J1) ok = wait_u(j) && ok;
#pragma unroll
        for (int k = 0; k < Q - 1; k++) q0[k] = q0[k + 1];
        q0[Q - 1] = j < J1 ? *reinterpret_cast<const float4 *>(ring + (j % NU) * plane_u + (r + M) * kBoxW +
                                                                kSideHalo + 4 * qc)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 v1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j >= 2 * M && j < J1) {
            const int ja = j - 2 * M;
            ok = wait_a(ja) && ok;
            if (ok && active) {
                const float *pc = ring + ((j - M) % NU) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc;
                const float *pa = aux1 + (ja % NA) * 3 * plane_a + r * kTileW + 4 * qc;
                const float4 um4 = *reinterpret_cast<const float4 *>(pa);
                const float4 c4 = *reinterpret_cast<const float4 *>(pa + plane_a);
                const float4 d4 = *reinterpret_cast<const float4 *>(pa + 2 * plane_a);
                const float umv[4] = {um4.x, um4.y, um4.z, um4.w};
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
                float res[4];
                update4<M, E, Q>(pc, q0, umv, cv, dv, cf, res);
                if (nsrc > 0) inject4(res, cv, s_src, s_sstart, ja, r, qc, src_row1);
                store4(out1, a, ja, row0 + r, col0 + 4 * qc, res);
                v1 = make_float4(res[0], res[1], res[2], res[3]);
            }
        }
#pragma unroll
        for (int k = 0; k < Q - 1; k++) q1[k] = q1[k + 1];
        q1[Q - 1] = v1;

        // stage 2: u^{n+2} at plane j - 2M - L
        if (j >= 2 * M + L) {
            const int jb = j - 2 * M - L;
            ok = wait_b(jb) && ok;
            if (ok && active) {
                const float *pc = box + (jb & 1) * plane_u + (r + M) * kBoxW + kSideHalo + 4 * qc;
                const float *pa = aux2 + (jb & 1) * 2 * plane_a + r * kTileW + 4 * qc;
                const float4 c4 = *reinterpret_cast<const float4 *>(pa);
                const float4 d4 = *reinterpret_cast<const float4 *>(pa + plane_a);
                const float umv[4] = {q0[0].x, q0[0].y, q0[0].z, q0[0].w};
                const float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
                float res[4];
                update4<M, 0, Q>(pc, q1, umv, cv, dv, cf, res);
                if (nsrc > 0) inject4(res, cv, s_src, s_sstart, jb, r, qc, src_row2);
                store4(out2, a, jb, row0 + r, col0 + 4 * qc, res);
            }
        }

        const bool wrote1 = j >= 2 * M && j < J1;
        if (wrote1) fence_proxy_async_global();  // u^{n+1} is read back through TMA
        if (!ok) *abort_flag = 1;
        // the ring slots read above are refilled by TMA (async proxy) after
        // this barrier: fence the generic-proxy reads against that
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (*abort_flag) {
            stop = true;
            break;
        }
        // the release orders every thread's stores of this plane (they
        // happen before it through the barrier) before the flag
        if (tid == 0 && wrote1) st_release(progress + tile, j - 2 * M + 1);
    }

    if (stop) {
        // record the error (unless one is recorded already), then drain the
        // copies this CTA issued, under one shared deadline
        if (tid == 0) {
            atomicCAS(status, 0, (int)FD_ERR_TIMEOUT);
            const unsigned long long deadline = global_ns() + kWaitLimitNs;
            for (int i = j; i <= issued1; i++) {
                mbar_wait_until(bar(i % NU), (uint32_t)((i / NU) & 1), deadline);
                if (i >= 2 * M) {
                    const int ia = i - 2 * M;
                    mbar_wait_until(bar(NU + ia % NA), (uint32_t)((ia / NA) & 1), deadline);
                }
            }
            for (int i = j > 2 * M + L ? j : 2 * M + L; i <= issued2; i++) {
                const int ib = i - 2 * M - L;
                mbar_wait_until(bar(NU + NA + (ib & 1)), (uint32_t)((ib >> 1) & 1), deadline);
            }
        }
        __syncthreads();
    }
}

template <int M>
cudaError_t configure_pair(size_t smem)
{
    return cudaFuncSetAttribute(acoustic_pair_kernel<M, kPairStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
}

template <int M>
int pair_occupancy(int threads, size_t smem)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, acoustic_pair_kernel<M, kPairStages>, threads, smem) !=
        cudaSuccess)
        return 0;
    return occ;
}

// threads of a CTA: 16 per row, whole warps (warp 0 polls with full-warp
// reductions; the extra lanes own no points)
int pair_threads(int rows_max) { return (16 * rows_max + 31) / 32 * 32; }

int occupancy_of(int M, int threads, size_t smem)
{
    switch (M) {
    case 2: return pair_occupancy<2>(threads, smem);
    case 3: return pair_occupancy<3>(threads, smem);
    case 4: return pair_occupancy<4>(threads, smem);
    }
    return 0;
}

}  // namespace

fd_status pair_plan_build(PairPlan &plan, int space_order, const Geom &g, float *const slot[2], float *c, float *d)
{
    const int want_rows = plan.force_rows;
    plan.ready = false;
    const int M = space_order / 2;
    if (g.ndim != 3 || M < 2 || M > 4) return FD_OK;
    if (g.n[0] > (1 << 30) || g.n[1] > (1 << 30) || g.n[2] > (1 << 30)) return FD_OK;
    int dev = 0, sms = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return set_error(FD_ERR_CUDA, "cudaGetDevice failed");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (sms <= 0 || smem_max <= 0) return set_error(FD_ERR_CUDA, "device attributes unavailable");
    cudaError_t e = cudaErrorInvalidValue;
    switch (M) {
    case 2: e = configure_pair<2>((size_t)smem_max); break;
    case 3: e = configure_pair<3>((size_t)smem_max); break;
    case 4: e = configure_pair<4>((size_t)smem_max); break;
    }
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "two-step kernel configuration: %s", cudaGetErrorString(e));

    TileArgs a{};
    a.n0 = (int)g.n[0];
    a.n1 = (int)g.n[1];
    a.n2 = (int)g.n[2];
    a.s0 = g.s0;
    a.s1 = g.s1;
    a.k2 = (a.n2 + kTileW - 1) / kTileW;
    a.kz = 1;
    a.stall_plane = -1;
    // Every column is resident at once, so the busiest SM sweeps
    // ceil(columns / SMs) columns of rows_max + M row-planes (the halo rows
    // come from L2 at about half the cost of a row): take the strip count
    // that minimises that, among those whose columns all fit; ties go to
    // fewer columns.
    const size_t reserve = 16 * 1024;  // shared memory kept for fused point lists
    int best_k1 = -1;
    double best_cost = 0;
    const int k1_lo = want_rows > 0 ? (a.n1 + want_rows - 1) / want_rows : (a.n1 + kPairMaxRows - 1) / kPairMaxRows;
    const int k1_hi = want_rows > 0 ? k1_lo : a.n1;
    for (int k1 = k1_lo; k1 <= k1_hi; k1++) {
        const int rows_max = (a.n1 + k1 - 1) / k1;
        if (rows_max > kPairMaxRows) continue;
        // a haloed box reaches M rows into the strips above and below: every
        // strip must be at least M rows tall so that it only reaches the
        // adjacent columns, the ones whose progress is checked
        if (k1 > 1 && a.n1 / k1 < M) break;
        const long long cols = (long long)k1 * a.k2;
        const size_t smem = pair_smem_layout(M, kPairStages, rows_max, 0, a.n0).end;
        if (smem + reserve > (size_t)smem_max) continue;
        if (cols > 8LL * sms) break;
        const int occ = occupancy_of(M, pair_threads(rows_max), smem);
        if (occ < 1 || cols > (long long)sms * occ) continue;
        const double cost = (double)((cols + sms - 1) / sms) * (rows_max + 0.5 * M);
        if (best_k1 < 0 || cost < best_cost - 1e-9) {
            best_k1 = k1;
            best_cost = cost;
        }
    }
    if (best_k1 < 0) {
        if (want_rows > 0) return set_error(FD_ERR_UNSUPPORTED, "two-step tiling: %d rows do not fit", want_rows);
        return FD_OK;
    }
    a.k1 = best_k1;
    a.rows_max = (a.n1 + a.k1 - 1) / a.k1;
    a.box_h = a.rows_max + 2 * M;

    plan.M = M;
    plan.stages = kPairStages;
    plan.args = a;
    plan.threads = pair_threads(a.rows_max);
    plan.smem = pair_smem_layout(M, kPairStages, a.rows_max, 0, a.n0).end;
    plan.smem_max = (size_t)smem_max;
    plan.slot[0] = slot[0];
    plan.slot[1] = slot[1];
    for (int s = 0; s < 2; s++) {
        fd_status st = tma_encode_3d(&plan.u_halo[s], slot[s], a, kBoxW, a.box_h);
        if (st != FD_OK) return st;
        st = tma_encode_3d(&plan.u_tile[s], slot[s], a, kTileW, a.rows_max);
        if (st != FD_OK) return st;
    }
    fd_status st = tma_encode_3d(&plan.c_tile, c, a, kTileW, a.rows_max);
    if (st != FD_OK) return st;
    st = tma_encode_3d(&plan.d_tile, d, a, kTileW, a.rows_max);
    if (st != FD_OK) return st;
    if (plan.progress) cudaFree(plan.progress);
    plan.progress = nullptr;
    if (cudaMalloc((void **)&plan.progress, sizeof(int) * (size_t)a.k1 * a.k2) != cudaSuccess)
        return set_error(FD_ERR_NOMEM, "two-step progress flags");
    plan.ready = true;
    return FD_OK;
}

fd_status pair_sparse_build(PairPlan &plan, const SparseHostView *src, cudaStream_t st)
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
    plan.smem = pair_smem_layout(plan.M, plan.stages, a.rows_max, 0, a.n0).end;
    if (!src || src->npoint <= 0) return FD_OK;
    std::vector<SrcEntry> all;
    std::vector<int> off;
    int max_s = 0, max_col = 0;
    fused_corner_lists(a, 1, src, all, off, max_s, max_col);  // one CTA per whole column
    const size_t smem = pair_smem_layout(plan.M, plan.stages, a.rows_max, max_s, a.n0).end;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the corners must not cost the co-residency of the columns
    if (smem > plan.smem_max ||
        (long long)a.k1 * a.k2 > (long long)sms * occupancy_of(plan.M, plan.threads, smem))
        return FD_OK;
    fd_status s = fused_upload(all, off, st, plan.fused, plan.fused_mem);
    if (s != FD_OK) return s;
    plan.has_src = true;
    plan.src_cap = max_s;
    plan.smem = smem;
    return FD_OK;
}

void pair_plan_release(PairPlan &plan, cudaStream_t st)
{
    plan.ready = false;
    if (plan.fused_mem || plan.progress) cudaStreamSynchronize(st);
    if (plan.fused_mem) cudaFree(plan.fused_mem);
    if (plan.progress) cudaFree(plan.progress);
    plan.fused_mem = nullptr;
    plan.progress = nullptr;
    plan.fused = SparseFused();
    plan.has_src = false;
}

cudaError_t launch_acoustic_pair(const PairPlan &plan, const Coef &cf, int b, int *status, const float *src_row1,
                                 const float *src_row2, cudaStream_t st)
{
    const TileArgs &a = plan.args;
    const int prev = b ^ 1;
    const int cols = a.k1 * a.k2;
    cudaError_t e = cudaMemsetAsync(plan.progress, 0, sizeof(int) * (size_t)cols, st);
    if (e != cudaSuccess) return e;
    const bool src = plan.has_src && src_row1 && src_row2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cols);
    cfg.blockDim = dim3((unsigned)plan.threads);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const SrcEntry *tab = src ? plan.fused.src : nullptr;
    const int *off = src ? plan.fused.src_off : nullptr;
    const float *r1 = src ? src_row1 : nullptr;
    const float *r2 = src ? src_row2 : nullptr;
    switch (plan.M) {
#define CASE(MM)                                                                                              \
    case MM:                                                                                                  \
        e = cudaLaunchKernelEx(&cfg, acoustic_pair_kernel<MM, kPairStages>, plan.u_halo[b], plan.u_tile[prev], \
                               plan.c_tile, plan.d_tile, plan.u_halo[prev], plan.slot[prev], plan.slot[b], a, cf,   \
                               status, plan.progress, tab, off, r1, r2, plan.src_cap);                           \
        break;
        CASE(2) CASE(3) CASE(4)
#undef CASE
    default:
        return cudaErrorInvalidValue;
    }
    return e;
}

}  // namespace fdgb
