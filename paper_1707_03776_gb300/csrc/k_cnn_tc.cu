// The closure network's 3x3x3 convolution on the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators), the alternative to the mma.sync
// kernel of k_cnn.cu with the same inputs and outputs.
//
// Implicit GEMM per output line of 128 points (the MMA's M = 128 TMEM lanes
// along d2), tcgen05.mma.kind::f16 (BF16 in, FP32 accumulate in TMEM) with
// both operands in shared memory.  One thread issues an MMA about every 60
// cycles whatever its N, and an N = 16 MMA reads a 4 KB A tile for 65 kFLOP,
// so the kernel makes each MMA as wide as the 16 output channels allow:
//   * a persistent CTA per SM sweeps tile columns of 4 output rows x 128
//     points along d0; each input plane tile (6 rows x 130 points x 16
//     channels, zero outside the grid) arrives by two TMA copies into a
//     6-plane ring as K-major no-swizzle core matrices (channel half h of
//     tile point p at byte h * 12544 + p * 16), so that the A tile of input
//     line l with d2 shift c is the same layout started (l * 130 + c) * 16
//     bytes in.  A, re-read by every MMA, is most of the operand traffic
//     that bounds the kernel (measured: the tensor core's operand pipe 81 %
//     busy, its math 28 %); taller tile columns re-read less of it but
//     measured slower (6 rows: 5 % slower, 8 rows with a 5-plane ring: 9 %);
//   * the three d1 taps b of an (input plane a, shift c) are the N = 16 b + o
//     columns of one B operand, and output row r's accumulator sits at column
//     16 (3 - r): input line l then feeds rows l + 1, l, l - 1 through one
//     contiguous column range -- one MMA per input line, N = 48 inside the
//     tile and 16 or 32 at its edges, 54 per output plane, no work wasted;
//   * two issuing warps take alternate output planes, each with two
//     accumulator sets of 64 columns (a clearing MMA with zero operands
//     starts each);
//   * warps 0-3 read a set back with tcgen05.ld (lane = point), apply bias,
//     ReLU and the input-gradient mask, store BF16 (or the one FP32 channel)
//     and hand it back.
// The sum over taps runs in another order than the mma.sync kernel's, so the
// two agree to FP32 rounding, not bit for bit.  TMA loads, MMA completion
// (tcgen05.commit) and the epilogue are ordered by mbarriers whose waits are
// bounded: a wait that gives up records FD_ERR_TIMEOUT in the status word,
// every other role stops at its next wait, and each issuing thread drains its
// tensor-core work before the tensor memory is freed.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fd_internal.h"
#include "fd_internal_host.h"
#include "k_sweep.cuh"

namespace fdgb {
namespace {
using namespace tile_dev;

constexpr int kUC = 16;                               // channels per point
constexpr int kTR = 4;                                // output rows per tile column
constexpr int kTW = 128;                              // output points per line = MMA M = TMEM lanes
constexpr int kPW = kTW + 2;                          // input line with the d2 halo
constexpr int kInRows = kTR + 2;                      // input lines per plane tile
constexpr uint32_t kHalfBytes = (kInRows * kPW * 16 + 127) / 128 * 128;  // one channel half (the A LBO)
constexpr uint32_t kPlaneBytes = 2 * kHalfBytes;
constexpr uint32_t kTmaBytes = 2 * kInRows * kPW * 16;  // what the two copies of a plane deliver
constexpr int kSRing = 6;                             // input planes in shared memory
constexpr uint32_t kAccCols = kTR * 16;               // one accumulator set: row r at 16 (kTR - 1 - r)
// 2 issuers x 2 buffers, allocated as a power of two (at least 32 columns)
constexpr uint32_t kTmemCols = 4 * kAccCols <= 32 ? 32 : 4 * kAccCols <= 64 ? 64 : 4 * kAccCols <= 128 ? 128
                                 : 4 * kAccCols <= 256 ? 256 : 512;
// warps: 0-3 epilogue (TMEM lanes 32w..), 4 loader, 5-6 MMA issuers
constexpr int kWarpLoad = 4, kWarpMma = 5;
constexpr int kThreads = 32 * (kWarpMma + 2);
constexpr uint32_t kWCombBytes = 1536;                // per (a, c): [2 halves][48 n = 16 b + o][8 k] BF16
constexpr uint32_t kWOff = kSRing * kPlaneBytes;
constexpr uint32_t kZOff = kWOff + 9 * kWCombBytes;   // 4 KB of zeros: the clearing MMA's operands
constexpr uint32_t kBarOff = kZOff + 4096;
// mbarriers: full (plane landed, TMA), empty (both issuers done with a
// plane), done (an accumulator set's MMAs done), free (its 4 epilogue warps
// done), fin (final drain of each issuer)
constexpr int kFull = 0, kEmpty = kSRing, kDone = 2 * kSRing, kFree = kDone + 4, kFin = kFree + 4,
              kNBars = kFin + 2;
constexpr uint32_t kSmemU = kBarOff + 8 * kNBars + 16;
__host__ __device__ constexpr uint32_t bar_count(int i)
{
    return (i >= kEmpty && i < kDone) ? 2u : (i >= kFree && i < kFin) ? 4u : 1u;
}
static_assert(kPlaneBytes % 128 == 0 && kHalfBytes % 128 == 0 && kWOff % 128 == 0 && kZOff % 128 == 0,
              "TMA destinations and descriptors");
static_assert((kHalfBytes >> 4) < (1u << 14), "descriptor offset field");
static_assert(kSmemU <= 227 * 1024, "shared memory");

// The MMA of input line l (-1..kTR: tile lines y0 - 1 .. y0 + kTR) for one
// (plane a, shift c): the d1 taps b = 0, 1, 2 of its 16 output channels go
// to rows l + 1, l, l - 1 (those inside the tile), the N = 16 b + o columns
// of B; with row r's accumulator at 16 (kTR - 1 - r) they are one contiguous
// range.  Returns the range's first accumulator column, N and first B row.
struct LineMma {
    uint32_t dcol;
    uint32_t n;
    uint32_t brow;
};
__host__ __device__ constexpr LineMma line_mma(int l)
{
    return l == -1        ? LineMma{16u * (kTR - 1), 16u, 0u}
           : l == 0       ? LineMma{16u * (kTR - 2), 32u, 0u}
           : l == kTR - 1 ? LineMma{0u, 32u, 16u}
           : l == kTR     ? LineMma{0u, 16u, 32u}
                          : LineMma{16u * (uint32_t)(kTR - 2 - l), 48u, 0u};
}

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

// instruction descriptor: D F32, A and B BF16, both K-major, M = 128, N
__host__ __device__ constexpr uint32_t idesc_n(uint32_t n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// D[tmem] (+)= A[smem descriptor] * B[smem descriptor]
__device__ __forceinline__ void umma_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
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
    conv3d_umma_kernel(const __grid_constant__ CUtensorMap xmap, const uint4 *__restrict__ wpack,
                       const float *__restrict__ bias, int cout, const __nv_bfloat16 *__restrict__ mask, void *y,
                       UDims d, int *status)
{
    extern __shared__ __align__(1024) unsigned char usm[];
    const uint32_t ring = smem_addr(usm);
    const uint32_t wsm = ring + kWOff;
    const uint32_t zsm = ring + kZOff;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(usm + kBarOff);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(usm + kBarOff + 8 * kNBars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(usm + kBarOff + 8 * kNBars + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto BAR = [&](int i) { return smem_addr(&bars[i]); };

    for (int q = tid; q < 9 * (int)kWCombBytes / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(usm + kWOff)[q] = wpack[q];
    for (int q = tid; q < 4096 / 16; q += blockDim.x) reinterpret_cast<uint4 *>(usm + kZOff)[q] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&xmap)) : "memory");
        for (int i = 0; i < kNBars; i++) mbar_init(BAR(i), bar_count(i));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == kWarpLoad) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr((const void *)tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    proxy_fence();  // the weights and zeros (generic stores) are read by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int tiles2 = (d.n2 + kTW - 1) / kTW;
    const int tiles1 = (d.n1 + kTR - 1) / kTR;
    const long long total = (long long)tiles2 * tiles1 * d.n0;
    const long long q_lo = (long long)blockIdx.x * total / gridDim.x;
    const long long q_hi = (long long)(blockIdx.x + 1) * total / gridDim.x;
    // planes are counted over the CTA's whole share (a segment of nout output
    // planes reads nout + 2 input planes): input g -> shared slot g % kSRing;
    // output oq -> issuer oq & 1, its accumulator buffer (oq >> 1) & 1, i.e.
    // accumulator set 2 (oq & 1) + ((oq >> 1) & 1)
    auto fail = [&]() {
        *abort_flag = 1;
        atomicExch(status, (int)FD_ERR_TIMEOUT);
    };
    auto acc_set = [](unsigned oq) { return (int)(2u * (oq & 1u) + ((oq >> 1) & 1u)); };

    if (warp == kWarpLoad) {
        // loader: every input plane of the CTA's share, kSRing ahead at most
        if (lane == 0) {
            unsigned g = 0;
            bool ok = true;
            for (long long q = q_lo; q < q_hi && ok;) {
                const Seg sg = segment_at(q, q_hi, d, tiles2);
                const int nin = sg.ze - sg.zs + 2;
                for (int i = 0; i < nin && ok; i++, g++) {
                    const int slot = (int)(g % kSRing);
                    // both issuers are done with the slot's previous plane
                    if (g >= (unsigned)kSRing &&
                        !mbar_wait_or_abort(BAR(kEmpty + slot), ((g / kSRing) - 1u) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bar = BAR(kFull + slot);
                    mbar_expect_tx(bar, kTmaBytes);
                    const uint32_t dst = ring + (uint32_t)slot * kPlaneBytes;
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        asm volatile(
                            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                            " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst + (uint32_t)h * kHalfBytes),
                            "l"(reinterpret_cast<unsigned long long>(&xmap)), "r"(0), "r"(h), "r"(sg.x0 - 1),
                            "r"(sg.y0 - 1), "r"(sg.zs - 1 + i), "r"(bar)
                            : "memory");
                }
                q += sg.ze - sg.zs;
            }
            if (!ok) fail();
            // the last kSRing loads may not have been waited on by an issuer
            const unsigned long long deadline = global_ns() + kWaitLimitNs;
            for (unsigned k = (g > (unsigned)kSRing ? g - kSRing : 0u); k < g; k++)
                mbar_wait_until(BAR(kFull + (int)(k % kSRing)), (k / kSRing) & 1u, deadline);
        }
        __syncwarp();
    } else if (warp >= kWarpMma) {
        // issuer P takes the outputs oq with oq & 1 == P: a clearing MMA,
        // then per (plane a, shift c) one MMA per input line (N = 16..48)
        const int P = warp - kWarpMma;
        if (lane == 0) {
            unsigned g0 = 0, oq0 = 0;  // first input and first output of the segment
            bool ok = true;
            for (long long q = q_lo; q < q_hi && ok;) {
                const Seg sg = segment_at(q, q_hi, d, tiles2);
                const int nout = sg.ze - sg.zs, nin = nout + 2;
                // each input gets one empty-commit from each issuer, after that
                // issuer's last read of it (at once if it reads none of them)
                auto commit_inputs = [&](int lo, int hi) {
                    for (int i = lo; i <= hi; i++) umma_commit(BAR(kEmpty + (int)((g0 + (unsigned)i) % kSRing)));
                };
                int o = ((oq0 & 1u) == (unsigned)P) ? 0 : 1;
                if (o >= nout) commit_inputs(0, nin - 1);
                int c_next = 0;
                for (; o < nout && ok; o += 2) {
                    const unsigned oq = oq0 + (unsigned)o;
                    const int set = acc_set(oq);
                    // the epilogue has read this accumulator set back
                    if (oq >= 4 && !mbar_wait_or_abort(BAR(kFree + set), ((oq >> 2) - 1u) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint32_t pl[3];
                    for (int a = 0; a < 3 && ok; a++) {
                        const unsigned g = g0 + (unsigned)(o + a);
                        ok = mbar_wait_or_abort(BAR(kFull + (int)(g % kSRing)), (g / kSRing) & 1u, abort_flag);
                        pl[a] = ring + (uint32_t)(g % kSRing) * kPlaneBytes;
                    }
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)set * kAccCols;
                    // clear the set: zeros times zeros, accumulator overwritten
                    umma_ss(acc, umma_desc(zsm, 2048, 128), umma_desc(zsm, kAccCols * 16, 128), idesc_n(kAccCols), 0u);
#pragma unroll
                    for (int a = 0; a < 3; a++)
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const uint32_t wb = wsm + (uint32_t)((a * 3 + c) * kWCombBytes);
#pragma unroll
                            for (int l = -1; l <= kTR; l++) {
                                constexpr uint32_t lbo_b = 48 * 16;
                                const LineMma m = line_mma(l);
                                umma_ss(acc + m.dcol,
                                        umma_desc(pl[a] + (uint32_t)(((l + 1) * kPW + c) * 16), kHalfBytes, 128),
                                        umma_desc(wb + m.brow * 16u, lbo_b, 128), idesc_n(m.n), 1u);
                            }
                        }
                    umma_commit(BAR(kDone + set));
                    const int hi = (o + 2 < nout) ? o + 1 : nin - 1;
                    commit_inputs(c_next, hi);
                    c_next = hi + 1;
                }
                g0 += (unsigned)nin;
                oq0 += (unsigned)nout;
                q += nout;
            }
            if (!ok) fail();
            const unsigned long long deadline = global_ns() + kWaitLimitNs;
            umma_commit(BAR(kFin + P));
            mbar_wait_until(BAR(kFin + P), 0u, deadline);
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 = points x0+32w..
        unsigned oq = 0;
        bool ok = true;
        for (long long q = q_lo; q < q_hi && ok;) {
            const Seg sg = segment_at(q, q_hi, d, tiles2);
            for (int z = sg.zs; z < sg.ze; z++) {
                const int set = acc_set(oq);
                const bool got =
                    __all_sync(0xffffffffu, mbar_wait_or_abort(BAR(kDone + set), (oq >> 2) & 1u, abort_flag));
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int r = 0; r < kTR; r++) {
                    uint32_t v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)set * kAccCols + 16u * (kTR - 1 - r), v);
                    const int gy = sg.y0 + r, gx = sg.x0 + 32 * warp + lane;
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
                        for (int h2 = 0; h2 < 2; h2++) {
                            const uint4 m4 = mk[h2];
                            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                            for (int jj = 0; jj < 4; jj++) {
                                const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162 *>(&mw[jj]);
                                if (!(__low2float(m2) > 0.f)) f[h2 * 8 + 2 * jj] = 0.f;
                                if (!(__high2float(m2) > 0.f)) f[h2 * 8 + 2 * jj + 1] = 0.f;
                            }
                        }
                    }
                    if (OUT_F32) {
                        reinterpret_cast<float *>(y)[pt] = f[0];
                    } else {
                        uint32_t packed[8];
#pragma unroll
                        for (int jj = 0; jj < 8; jj++) {
                            const __nv_bfloat162 t2 = __floats2bfloat162_rn(f[2 * jj], f[2 * jj + 1]);
                            packed[jj] = *reinterpret_cast<const uint32_t *>(&t2);
                        }
                        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(y) + pt * kUC);
                        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                    }
                }
                // this set's values are in registers: hand it back
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(BAR(kFree + set));
                oq++;
            }
            q += sg.ze - sg.zs;
        }
        if (!ok && lane == 0) fail();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == kWarpLoad) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// weights w[27][cin][cout] (FP32) into the B operands: per (plane a, shift
// c), [2 halves][48 n][8 k] BF16 with n = 16 b + o (the three d1 taps side by
// side); flip = the input-gradient convolution (taps mirrored, channel axes
// exchanged)
__global__ void pack_umma_kernel(const float *__restrict__ w, int cin, int cout, int flip,
                                 __nv_bfloat16 *__restrict__ out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 9 * 768) return;
    const int comb = q / 768, rem = q % 768;
    const int h = rem / 384, n = (rem / 8) % 48, kk = rem % 8;
    const int a = comb / 3, c = comb % 3, b = n / 16, o = n % 16;
    const int t = a * 9 + b * 3 + c;
    const int k = h * 8 + kk;
    float v = 0.f;
    if (!flip) {
        if (k < cin && o < cout) v = w[((long long)t * cin + k) * cout + o];
    } else {
        if (k < cout && o < cin) v = w[((long long)(26 - t) * cin + o) * cout + k];
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
    pack_umma_kernel<<<(9 * 768 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, cin, cout, flip,
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
        auto k = conv3d_umma_kernel<R, M, F>;                                                             \
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
