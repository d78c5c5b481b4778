// The closure network's 3x3x3 convolution on the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators), the alternative to the mma.sync
// kernel of k_cnn.cu with the same inputs, outputs and results.
//
// Implicit GEMM per output line of 128 points (the MMA's M = 128 TMEM lanes
// along d2): D[128 x 16 channels] = sum over the 27 taps of A_tap[128 x 16]
// B_tap[16 x 16], one tcgen05.mma.kind::f16 (M = 128, N = 16, K = 16, BF16 in,
// FP32 accumulate) per tap.  With 16 output channels an MMA that takes its
// 4 KB A tile from shared memory is bound by those reads (4 KB per 65 kFLOP),
// so here the A operand lives in tensor memory:
//   * a persistent CTA per SM (all 512 TMEM columns) sweeps tile columns of
//     2 output rows x 128 points along d0; each input plane tile (4 rows x 130
//     points x 16 channels, zero outside the grid) arrives by two TMA copies
//     into a 6-plane shared-memory ring, laid out as K-major no-swizzle core
//     matrices (channel half h of tile point p at byte (h * 520 + p) * 16);
//   * tcgen05.cp copies each of its 4 input lines three times into a 4-plane
//     TMEM ring, started 0, 1 and 2 points in: the three d2 shifts of the
//     taps, so that lane i holds input point x0 + i - 1 + c for shift c;
//   * the 54 MMAs of an output plane (2 rows x 27 taps) then read A from TMEM
//     and only their 512-byte weight tile from shared memory, into one of two
//     accumulator buffers (2 rows x 16 columns);
//   * warps 0-3 read an accumulator buffer back with tcgen05.ld (lane =
//     point), apply bias, ReLU and the input-gradient mask, store BF16 (or the
//     one FP32 channel) and hand the buffer back; warp 4 issues everything.
// TMA loads, cp and MMA completion (tcgen05.commit) and the epilogue are
// ordered by mbarriers whose waits are bounded: a wait that gives up records
// FD_ERR_TIMEOUT in the status word, the other role stops at its next wait,
// and the CTA drains its copies and tensor-core work and frees the tensor
// memory before it leaves.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fd_internal.h"
#include "fd_internal_host.h"
#include "k_sweep.cuh"

namespace fdgb {
namespace {
using namespace tile_dev;

constexpr int kUC = 16;                               // channels per point
constexpr int kTR = 2;                                // output rows per tile column
constexpr int kTW = 128;                              // output points per line = MMA M = TMEM lanes
constexpr int kPW = kTW + 2;                          // input line with the d2 halo
constexpr int kInRows = kTR + 2;                      // input lines per plane tile
constexpr int kPts = kInRows * kPW;                   // points per input plane tile
constexpr uint32_t kHalfBytes = kPts * 16;            // one channel half of a tile (the A LBO)
constexpr uint32_t kPlaneBytes = 2 * kHalfBytes;
constexpr int kSRing = 6;                             // input planes in shared memory
constexpr int kTRing = 4;                             // input planes in tensor memory
constexpr uint32_t kPlaneCols = kInRows * 3 * 8;      // TMEM columns of an input plane (lines x shifts x K/2)
constexpr uint32_t kAccCol = kTRing * kPlaneCols;     // first accumulator column
constexpr uint32_t kTmemCols = 512;
constexpr int kThreads = 160;                         // warps 0-3: epilogue; warp 4: copies and MMAs
constexpr uint32_t kWTapBytes = 512;                  // [2 halves][16 n][8 k] BF16
constexpr uint32_t kWOff = kSRing * kPlaneBytes;
constexpr uint32_t kBarOff = kWOff + 27 * kWTapBytes;
constexpr int kNBars = 2 * kSRing + 5;                // full, empty, mma_done[2], acc_free[2], fin
constexpr uint32_t kSmemU = kBarOff + 8 * kNBars + 16;
static_assert(kAccCol + 2 * kTR * 16 <= kTmemCols, "tensor memory layout");
static_assert(kPlaneBytes % 128 == 0 && kHalfBytes % 128 == 0 && kWOff % 128 == 0, "TMA destinations");
static_assert((kHalfBytes >> 4) < (1u << 14), "descriptor offset field");

struct UDims {
    int n0, n1, n2;
};

// shared-memory matrix descriptor: no swizzle, start / leading / stride byte
// offsets in 16-byte units, descriptor version 1
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D F32, A and B BF16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// D[tmem] (+)= A[tmem] * B[smem descriptor]
__device__ __forceinline__ void umma_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

// 128 rows x 256 bits from shared memory (descriptor) into TMEM lanes 0..127
__device__ __forceinline__ void tmem_cp_128x256b(uint32_t taddr, uint64_t sdesc)
{
    asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Wait for phase `parity` of a barrier, giving up after kWaitLimitNs or as
// soon as the CTA's abort flag is raised by the other role.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

// The work of a CTA: the linear range [q_lo, q_hi) of (tile column, output
// plane) items, tile columns outermost; a segment is the run of it inside one
// tile column.
struct Seg {
    int x0, y0, zs, ze;
};

__device__ __forceinline__ Seg segment_at(long long q, long long q_hi, const UDims &d, int tiles2)
{
    const long long col = q / d.n0;
    const int zs = (int)(q - col * d.n0);
    const long long end = min(q_hi, (col + 1) * (long long)d.n0);
    Seg s;
    s.x0 = (int)(col % tiles2) * kTW;
    s.y0 = (int)(col / tiles2) * kTR;
    s.zs = zs;
    s.ze = zs + (int)(end - q);
    return s;
}

template <bool RELU, bool MASK, bool OUT_F32>
__global__ void __launch_bounds__(kThreads, 1)
    conv3d_tmem_kernel(const __grid_constant__ CUtensorMap xmap, const uint4 *__restrict__ wpack,
                       const float *__restrict__ bias, int cout, const __nv_bfloat16 *__restrict__ mask, void *y,
                       UDims d, int *status)
{
    extern __shared__ __align__(1024) unsigned char usm[];
    const uint32_t ring = smem_addr(usm);
    const uint32_t wsm = ring + kWOff;
    // barriers: full[kSRing] (plane landed), empty[kSRing] (its copies to
    // TMEM done), mma_done[2] (an accumulator buffer's MMAs done),
    // acc_free[2] (its epilogue done; 4 warp arrivals), fin (final drain)
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(usm + kBarOff);
    constexpr int kFull = 0, kEmpty = kSRing, kDone = 2 * kSRing, kFree = 2 * kSRing + 2, kFin = 2 * kSRing + 4;
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(usm + kBarOff + 8 * kNBars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(usm + kBarOff + 8 * kNBars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto BAR = [&](int i) { return smem_addr(&bars[i]); };

    for (int q = tid; q < 27 * (int)kWTapBytes / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(usm + kWOff)[q] = wpack[q];
    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&xmap)) : "memory");
        for (int i = 0; i < kNBars; i++) mbar_init(BAR(i), (i == kFree || i == kFree + 1) ? 4u : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr((const void *)tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    proxy_fence();  // the weights (generic stores) are read by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int tiles2 = (d.n2 + kTW - 1) / kTW;
    const int tiles1 = (d.n1 + kTR - 1) / kTR;
    const long long total = (long long)tiles2 * tiles1 * d.n0;
    const long long q_lo = (long long)blockIdx.x * total / gridDim.x;
    const long long q_hi = (long long)(blockIdx.x + 1) * total / gridDim.x;

    if (warp == 4) {
        if (lane == 0) {
            unsigned g_load = 0, g_full = 0;  // plane loads issued / whose arrival was waited (in order)
            unsigned oq = 0;                  // output planes whose MMAs were issued
            bool ok = true;
            const uint64_t bdesc0 = umma_desc(wsm, 256, 128);
            for (long long q = q_lo; q < q_hi && ok;) {
                const Seg sg = segment_at(q, q_hi, d, tiles2);
                const int nout = sg.ze - sg.zs, nin = nout + 2;
                const unsigned load0 = g_load, oq0 = oq;
                // input i of the segment is plane zs - 1 + i: shared slot
                // (load0 + i) % kSRing, TMEM slot i % kTRing
                auto load = [&](int i) -> bool {
                    const unsigned g = load0 + (unsigned)i;
                    const int slot = (int)(g % kSRing);
                    // the slot's previous plane has been copied to TMEM
                    if (g >= (unsigned)kSRing &&
                        !mbar_wait_or_abort(BAR(kEmpty + slot), ((g / kSRing) - 1u) & 1u, abort_flag))
                        return false;
                    const uint32_t bar = BAR(kFull + slot);
                    mbar_expect_tx(bar, kPlaneBytes);
                    const uint32_t dst = ring + (uint32_t)slot * kPlaneBytes;
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        asm volatile(
                            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst + (uint32_t)h * kHalfBytes),
                            "l"(reinterpret_cast<unsigned long long>(&xmap)), "r"(0), "r"(h), "r"(sg.x0 - 1),
                            "r"(sg.y0 - 1), "r"(sg.zs - 1 + i), "r"(bar)
                            : "memory");
                    g_load++;
                    return true;
                };
                auto cp_in = [&](int i) -> bool {
                    const unsigned g = load0 + (unsigned)i;
                    const int slot = (int)(g % kSRing);
                    if (!mbar_wait_or_abort(BAR(kFull + slot), (g / kSRing) & 1u, abort_flag)) return false;
                    g_full++;
                    tc_fence_after();
                    const uint32_t src = ring + (uint32_t)slot * kPlaneBytes;
                    const uint32_t tcol = tmem + (uint32_t)(i % kTRing) * kPlaneCols;
#pragma unroll
                    for (int r = 0; r < kInRows; r++)
#pragma unroll
                        for (int c = 0; c < 3; c++)
                            tmem_cp_128x256b(tcol + (uint32_t)((r * 3 + c) * 8),
                                             umma_desc(src + (uint32_t)((r * kPW + c) * 16), kHalfBytes, 128));
                    umma_commit(BAR(kEmpty + slot));
                    return true;
                };
                const int npre = nin < kSRing ? nin : kSRing;
                for (int i = 0; i < npre && ok; i++) ok = load(i);
                for (int i = 0; i < 3 && ok; i++) ok = cp_in(i);
                int next_load = npre, next_cp = 3;
                for (int o = 0; o < nout && ok; o++) {
                    const unsigned b = oq & 1u;
                    // the epilogue has read this accumulator buffer back
                    if (oq >= 2 && !mbar_wait_or_abort(BAR(kFree + b), ((oq >> 1) - 1u) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dcol = tmem + kAccCol + b * 32u;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        const uint32_t pl = tmem + (uint32_t)((o + a) % kTRing) * kPlaneCols;
#pragma unroll
                        for (int bb = 0; bb < 3; bb++)
#pragma unroll
                            for (int c = 0; c < 3; c++) {
                                const int t = a * 9 + bb * 3 + c;
#pragma unroll
                                for (int ro = 0; ro < kTR; ro++)
                                    umma_tmem_a(dcol + (uint32_t)(ro * 16), pl + (uint32_t)(((ro + bb) * 3 + c) * 8),
                                                bdesc0 + (uint64_t)(t * (kWTapBytes >> 4)), t > 0 ? 1u : 0u);
                            }
                    }
                    umma_commit(BAR(kDone + b));
                    oq++;
                    if (next_cp < nin) {
                        // the TMEM slot of input next_cp - kTRing is free
                        // once the last output reading it (that index) is done
                        if (next_cp >= kTRing) {
                            const unsigned ow = oq0 + (unsigned)(next_cp - kTRing);
                            if (!mbar_wait_or_abort(BAR(kDone + (ow & 1u)), (ow >> 1) & 1u, abort_flag)) {
                                ok = false;
                                break;
                            }
                        }
                        if (!cp_in(next_cp++)) {
                            ok = false;
                            break;
                        }
                    }
                    if (next_load < nin && !load(next_load++)) {
                        ok = false;
                        break;
                    }
                }
                // the segment's last commit covers every copy and MMA of it:
                // afterwards all TMEM and shared slots are free
                if (ok && oq > oq0) {
                    const unsigned ow = oq - 1;
                    ok = mbar_wait_or_abort(BAR(kDone + (ow & 1u)), (ow >> 1) & 1u, abort_flag);
                }
                q += nout;
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(status, (int)FD_ERR_TIMEOUT);
            }
            // drain: plane copies still owed, then every tcgen05 operation
            // issued (one more commit), under one shared deadline
            const unsigned long long deadline = global_ns() + kWaitLimitNs;
            for (unsigned g = g_full; g < g_load; g++)
                mbar_wait_until(BAR(kFull + (int)(g % kSRing)), (g / kSRing) & 1u, deadline);
            umma_commit(BAR(kFin));
            mbar_wait_until(BAR(kFin), 0u, deadline);
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 = points x0+32w..
        unsigned oq = 0;
        bool ok = true;
        for (long long q = q_lo; q < q_hi && ok;) {
            const Seg sg = segment_at(q, q_hi, d, tiles2);
            for (int z = sg.zs; z < sg.ze; z++) {
                const unsigned b = oq & 1u;
                const bool got =
                    __all_sync(0xffffffffu, mbar_wait_or_abort(BAR(kDone + b), (oq >> 1) & 1u, abort_flag));
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int ro = 0; ro < kTR; ro++) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + kAccCol + b * 32u + (uint32_t)(ro * 16), v);
                    const int gy = sg.y0 + ro, gx = sg.x0 + 32 * warp + lane;
                    if (gy >= d.n1 || gx >= d.n2) continue;
                    const long long pt = ((long long)z * d.n1 + gy) * d.n2 + gx;
                    float f[16];
#pragma unroll
                    for (int o = 0; o < 16; o++) {
                        float t = __uint_as_float(v[o]) + ((bias && o < cout) ? bias[o] : 0.f);
                        if (RELU) t = fmaxf(t, 0.f);
                        f[o] = t;
                    }
                    if (MASK) {
                        const uint4 *mk = reinterpret_cast<const uint4 *>(mask + pt * kUC);
#pragma unroll
                        for (int hh = 0; hh < 2; hh++) {
                            const uint4 m4 = mk[hh];
                            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                            for (int j = 0; j < 4; j++) {
                                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162 *>(&mw[j]);
                                if (!(__low2float(m2) > 0.f)) f[hh * 8 + 2 * j] = 0.f;
                                if (!(__high2float(m2) > 0.f)) f[hh * 8 + 2 * j + 1] = 0.f;
                            }
                        }
                    }
                    if (OUT_F32) {
                        reinterpret_cast<float *>(y)[pt] = f[0];
                    } else {
                        uint32_t packed[8];
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const __nv_bfloat162 t2 = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
                            packed[j] = *reinterpret_cast<const uint32_t *>(&t2);
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(y) + pt * kUC);
                        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                    }
                }
                // this buffer's values are in registers: hand it back
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(BAR(kFree + b));
                oq++;
            }
            q += sg.ze - sg.zs;
        }
        if (!ok && lane == 0) {
            *abort_flag = 1;
            atomicExch(status, (int)FD_ERR_TIMEOUT);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 4) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// weights w[27][cin][cout] (FP32) into [27][2 halves][16 n][8 k] BF16; flip =
// the input-gradient convolution (taps mirrored, channel axes exchanged)
__global__ void pack_umma_kernel(const float *__restrict__ w, int cin, int cout, int flip,
                                 __nv_bfloat16 *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 27 * 256) return;
    const int t = q / 256, rem = q % 256;
    const int h = rem / 128, n = (rem / 8) % 16, kk = rem % 8;
    const int k = h * 8 + kk;
    float v = 0.f;
    if (!flip) {
        if (k < cin && n < cout) v = w[((long long)t * cin + k) * cout + n];
    } else {
        if (k < cout && n < cin) v = w[((long long)(26 - t) * cin + n) * cout + k];
    }
    out[q] = __float2bfloat16(v);
}

}  // namespace
}  // namespace fdgb

using namespace fdgb;

extern "C" fd_status fd_cnn_pack_weights_tc(const float *w, int cin, int cout, int flip, void *out, void *stream)
{
    if (!w || !out || cin < 1 || cin > 16 || cout < 1 || cout > 16)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_pack_weights_tc: bad arguments");
    pack_umma_kernel<<<(27 * 256 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, cin, cout, flip,
                                                                              (__nv_bfloat16 *)out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_cnn_pack_weights_tc: %s", cudaGetErrorString(e));
    return FD_OK;
}

namespace {
typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeFn get_encode()
{
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    }
    return fn;
}
}  // namespace

extern "C" fd_status fd_cnn_conv3d_tc(const int64_t *shape, const void *x, const void *wpack, const float *bias,
                                      int cout, int relu, const void *mask, void *y, int y_fp32, int *status,
                                      void *stream)
{
    using namespace fdgb;
    if (!shape || !x || !wpack || !y || !status || cout < 1 || cout > 16)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_conv3d_tc: bad arguments");
    for (int a = 0; a < 3; a++)
        if (shape[a] < 1 || shape[a] > (1 << 20)) return set_error(FD_ERR_INVALID_ARG, "fd_cnn_conv3d_tc: bad shape");
    if (y_fp32 && (cout != 1 || relu || mask))
        return set_error(FD_ERR_UNSUPPORTED, "fd_cnn_conv3d_tc: FP32 output is one linear channel");
    if (((uintptr_t)x & 15) != 0 || ((uintptr_t)y & 15) != 0 || ((uintptr_t)mask & 15) != 0)
        return set_error(FD_ERR_LAYOUT, "fd_cnn_conv3d_tc: buffers must be 16-byte aligned");
    UDims d{(int)shape[0], (int)shape[1], (int)shape[2]};
    // activations as a 5D BF16 tensor (8 channels, 2 halves, n2, n1, n0)
    CUtensorMap map;
    cuuint64_t dims[5] = {8, 2, (cuuint64_t)d.n2, (cuuint64_t)d.n1, (cuuint64_t)d.n0};
    cuuint64_t strides[4] = {16, 32, 32ull * d.n2, 32ull * d.n2 * d.n1};
    cuuint32_t box[5] = {8, 1, (cuuint32_t)kPW, (cuuint32_t)kInRows, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    EncodeFn enc = get_encode();
    if (!enc) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_error(FD_ERR_CUDA, "fd_cnn_conv3d_tc: tensor map encoding failed");
    // persistent: one CTA per SM (each holds all of its SM's tensor memory),
    // each taking an equal share of the (tile column, plane) items
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            return set_error(FD_ERR_CUDA, "fd_cnn_conv3d_tc: device query failed");
    }
    const long long items = (long long)((d.n2 + kTW - 1) / kTW) * ((d.n1 + kTR - 1) / kTR) * d.n0;
    dim3 grid((unsigned)(items < sms ? items : sms));
    cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16 *mk = (const __nv_bfloat16 *)mask;
    const uint4 *wp = (const uint4 *)wpack;
    cudaError_t e = cudaSuccess;
#define LAUNCH(R, M, F)                                                                                   \
    do {                                                                                                  \
        auto k = conv3d_tmem_kernel<R, M, F>;                                                             \
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemU);            \
        if (e == cudaSuccess) {                                                                           \
            k<<<grid, kThreads, kSmemU, st>>>(map, wp, bias, cout, mk, y, d, status);                     \
            e = cudaGetLastError();                                                                       \
        }                                                                                                 \
    } while (0)
    if (y_fp32) LAUNCH(false, false, true);
    else if (relu && mask) LAUNCH(true, true, false);
    else if (relu) LAUNCH(true, false, false);
    else if (mask) LAUNCH(false, true, false);
    else LAUNCH(false, false, false);
#undef LAUNCH
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_cnn_conv3d_tc: %s", cudaGetErrorString(e));
    return FD_OK;
}
