// The closure network's 3x3x3 convolution on the 5th-generation tensor cores
// (tcgen05.mma with TMEM accumulators), the alternative to the mma.sync
// kernel of k_cnn.cu with the same inputs, outputs and results.
//
// Implicit GEMM per output row of 128 points: D[128 points x 16 channels] =
// sum over the 27 taps of A_tap[128 x 16] B_tap[16 x 16], one
// tcgen05.mma.kind::f16 (M = 128, N = 16, K = 16, BF16 in, FP32 accumulate)
// per tap, issued by one thread; the accumulators (2 rows x 16 columns, two
// buffers by plane parity) live in tensor memory and are read back with
// tcgen05.ld by the 4 warps (lane = point).  A CTA owns 2 rows x 128 points and
// sweeps 16 planes along d0; each input plane (4 rows x 130 points with the
// halo) arrives by two TMA copies of a 5D view of the activations (8 channels,
// 2 halves, n2, n1, n0) -- zero outside the grid -- into a 5-plane ring, laid
// out as the K-major no-swizzle core matrices of the A operand: channel half h
// of plane point p at byte (h * points + p) * 16, so a tap's A tile is the
// same layout started (p_tap * 16) bytes in (descriptor LBO = the half stride,
// SBO = 128).  Weights: [27][2 halves][16 n][8 k] BF16 (LBO 256, SBO 128).
// Plane loads, MMA completion (tcgen05.commit) and the epilogue are ordered by
// mbarriers whose waits are bounded: a wait that gives up records
// FD_ERR_TIMEOUT in the status word, drains what is still in flight and frees
// the tensor memory before the CTA leaves.
//
// With only 16 output channels every MMA reads a 4 KB A tile for 65 kFLOP,
// so the tensor core is bound by its shared-memory operand reads (measured:
// tensor pipe 77 % busy at ~190 TFLOP/s), no faster per point than the
// mma.sync kernel, which therefore remains the closure's path.
#include <cuda_bf16.h>
#include <stdint.h>

#include "fd_internal.h"
#include "fd_internal_host.h"
#include "k_sweep.cuh"

namespace fdgb {
namespace {
using namespace tile_dev;

constexpr int kUC = 16;                   // channels per point
constexpr int kUTR = 2;                   // output rows per CTA
constexpr int kUW = 128;                  // output points per row = MMA M
constexpr int kUPW = kUW + 2;             // plane row with the halo
constexpr int kUPts = (kUTR + 2) * kUPW;  // points per plane
constexpr int kURing = 5;                 // planes held
constexpr int kUZc = 16;                  // planes per CTA
constexpr int kUThreads = 128;            // 4 warps: TMEM lanes 0..127
constexpr uint32_t kUTmemCols = 64;       // 2 accumulator buffers x kUTR x 16 columns
constexpr uint32_t kPlaneBytes = kUPts * kUC * 2;
constexpr uint32_t kWTapBytes = 512;      // [2 halves][16 n][8 k] BF16
constexpr uint32_t kSmemU = kURing * kPlaneBytes + 27 * kWTapBytes + 8 * (kURing + 4);

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

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
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

template <bool RELU, bool MASK, bool OUT_F32>
__global__ void __launch_bounds__(kUThreads, 2)
    conv3d_umma_kernel(const __grid_constant__ CUtensorMap xmap, const uint4 *__restrict__ wpack,
                       const float *__restrict__ bias, int cout, const __nv_bfloat16 *__restrict__ mask, void *y,
                       UDims d, int *status)
{
    extern __shared__ __align__(1024) unsigned char usm[];
    const uint32_t ring = smem_addr(usm);
    const uint32_t wsm = ring + kURing * kPlaneBytes;
    // barriers: full[kURing] (plane landed), done[2] (MMAs of a plane parity)
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(usm + kURing * kPlaneBytes + 27 * kWTapBytes);
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(bars + kURing + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + kURing + 3);

    const int tiles2 = (d.n2 + kUW - 1) / kUW;
    const int col0 = (blockIdx.x % tiles2) * kUW;
    const int row0 = (blockIdx.x / tiles2) * kUTR;
    const int z0 = blockIdx.y * kUZc;
    const int z1 = min(d.n0, z0 + kUZc);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int q = tid; q < 27 * (int)kWTapBytes / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(usm + kURing * kPlaneBytes)[q] = wpack[q];
    if (tid == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&xmap)) : "memory");
        for (int i = 0; i < kURing + 2; i++) mbar_init(smem_addr(&bars[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr((const void *)tmem_slot)),
                     "r"(kUTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    proxy_fence();  // the weights (generic stores) are read by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // plane z -> ring slot z % kURing: both channel halves by TMA (zero outside)
    unsigned loads_into[kURing];
    for (int i = 0; i < kURing; i++) loads_into[i] = 0;
    auto issue_plane = [&](int z) {
        const int slot = ((z % kURing) + kURing) % kURing;
        const uint32_t bar = smem_addr(&bars[slot]);
        const uint32_t dst = ring + (uint32_t)slot * kPlaneBytes;
        mbar_expect_tx(bar, kPlaneBytes);
        for (int h = 0; h < 2; h++)
            asm volatile(
                "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst + (uint32_t)(h * kUPts * 16)),
                "l"(reinterpret_cast<unsigned long long>(&xmap)), "r"(0), "r"(h), "r"(col0 - 1), "r"(row0 - 1),
                "r"(z), "r"(bar)
                : "memory");
        loads_into[slot]++;
    };
    unsigned waited_full[kURing];
    for (int i = 0; i < kURing; i++) waited_full[i] = 0;
    auto wait_plane = [&](int z) {
        const int slot = ((z % kURing) + kURing) % kURing;
        const bool r = mbar_wait_bounded(smem_addr(&bars[slot]), waited_full[slot] & 1u);
        if (r) waited_full[slot]++;  // a copy that did not land is still owed
        return r;
    };
    if (tid == 0) {
        issue_plane(z0 - 1);
        issue_plane(z0);
        issue_plane(z0 + 1);
    }

    unsigned waited[2] = {0u, 0u};
    int issued_planes = 0;
    bool ok = true;
    // A descriptor offsets (16-byte units) of tap (b, c) and row r within a plane
    const uint64_t lbo_sbo = ((uint64_t)((kUPts * 16u) >> 4) << 16) | ((uint64_t)(128u >> 4) << 32) | ((uint64_t)1 << 46);
    const uint64_t bdesc0 = ((uint64_t)((wsm >> 4) & 0x3FFFu)) | ((uint64_t)(256u >> 4) << 16) |
                            ((uint64_t)(128u >> 4) << 32) | ((uint64_t)1 << 46);

    auto epilogue = [&](int p) {
        const int b = p & 1;
        const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(&bars[kURing + b]), waited[b] & 1u));
        if (!got) {
            ok = false;
            return;
        }
        waited[b]++;
        tc_fence_after();
#pragma unroll
        for (int r = 0; r < kUTR; r++) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * kUTR * 16 + r * 16), v);
            const int gy = row0 + r, gx = col0 + 32 * warp + lane;
            if (gy >= d.n1 || gx >= d.n2) continue;
            const long long pt = ((long long)p * d.n1 + gy) * d.n2 + gx;
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
        tc_fence_before();
    };

    for (int z = z0; z < z1; z++) {
        // every warp is done with the TMEM buffer the MMAs below overwrite
        // (its epilogue ran two planes ago) and with nothing else
        __syncthreads();
        if (*abort_flag) break;
        if (tid == 0) {
            // plane z+2 goes where plane z-3 was: its last readers (the MMAs
            // of plane z-2) finished before the epilogue of z-2
            issue_plane(z + 2);
            bool good = true;
            if (z == z0) good = wait_plane(z - 1) && wait_plane(z);
            good = good && wait_plane(z + 1);
            if (!good) {
                *abort_flag = 1;
            } else {
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)((z & 1) * kUTR * 16);
                uint64_t adesc_plane[3];
#pragma unroll
                for (int a = 0; a < 3; a++)
                    adesc_plane[a] = lbo_sbo |
                                     (uint64_t)(((ring + (uint32_t)((z - 1 + a + kURing) % kURing) * kPlaneBytes) >> 4) &
                                                0x3FFFu);
#pragma unroll
                for (int t = 0; t < 27; t++) {
                    const int a = t / 9, bb = (t / 3) % 3 - 1, c = t % 3 - 1;
                    const uint64_t bdesc = bdesc0 + (uint64_t)(t * (kWTapBytes >> 4));
#pragma unroll
                    for (int r = 0; r < kUTR; r++) {
                        const uint32_t off = (uint32_t)((r + 1 + bb) * kUPW + 1 + c);  // points = 16-byte units
                        umma_bf16(acc + (uint32_t)(r * 16), adesc_plane[a] + off, bdesc, t > 0 ? 1u : 0u);
                    }
                }
                umma_commit(smem_addr(&bars[kURing + (z & 1)]));
            }
        }
        __syncthreads();
        if (*abort_flag) break;
        issued_planes++;
        if (z > z0) epilogue(z - 1);
        if (!ok) *abort_flag = 1;
    }
    if (ok && !*abort_flag && z1 > z0) epilogue(z1 - 1);
    // after a wait gave up, every barrier still owed is waited on under one
    // shared deadline, so one that never completes does not stop the drain
    // short of the others
    const bool aborted = !ok || *abort_flag;
    const unsigned long long deadline = global_ns() + kWaitLimitNs;
    if (aborted) {
        if (tid == 0) atomicExch(status, (int)FD_ERR_TIMEOUT);
        for (int b = 0; b < 2; b++) {
            const unsigned owed = (unsigned)((issued_planes + (b == 0 ? 1 : 0)) / 2);
            while (waited[b] < owed) {
                if (!mbar_wait_until(smem_addr(&bars[kURing + b]), waited[b] & 1u, deadline)) break;
                waited[b]++;
            }
        }
    }
    // the TMA copies still owed (planes issued but never consumed)
    if (tid == 0)
        for (int i = 0; i < kURing; i++)
            while (waited_full[i] < loads_into[i]) {
                if (!mbar_wait_until(smem_addr(&bars[i]), waited_full[i] & 1u, deadline)) break;
                waited_full[i]++;
            }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kUTmemCols));
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
    cuuint32_t box[5] = {8, 1, (cuuint32_t)kUPW, (cuuint32_t)(kUTR + 2), 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    EncodeFn enc = get_encode();
    if (!enc) return set_error(FD_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return set_error(FD_ERR_CUDA, "fd_cnn_conv3d_tc: tensor map encoding failed");
    dim3 grid((unsigned)(((d.n2 + kUW - 1) / kUW) * ((d.n1 + kUTR - 1) / kUTR)), (unsigned)((d.n0 + kUZc - 1) / kUZc));
    cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16 *mk = (const __nv_bfloat16 *)mask;
    const uint4 *wp = (const uint4 *)wpack;
    cudaError_t e = cudaSuccess;
#define LAUNCH(R, M, F)                                                                                   \
    do {                                                                                                  \
        auto k = conv3d_umma_kernel<R, M, F>;                                                             \
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemU);            \
        if (e == cudaSuccess) {                                                                           \
            k<<<grid, kUThreads, kSmemU, st>>>(map, wp, bias, cout, mk, y, d, status);                    \
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
