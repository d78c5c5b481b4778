// Kernels of the learned closure: a 4-layer 3x3x3 CNN that corrects the
// coarse-grid update.
//
// Activations are channels-last BF16, 16 channels per point (32 bytes;
// channel counts below 16 are zero-padded).  The convolution is an implicit
// GEMM on the tensor cores: per output point (GEMM row) and output channel
// (column), K = 27 taps x 16 input channels, issued as one mma.sync
// m16n8k16 (BF16 in, FP32 accumulate) per tap, 16 points and 8 output
// channels.  A CTA owns 8 rows x 64 points of a d1-d2 tile and streams d0,
// keeping the three input planes a tap reaches (plus one in flight) in shared
// memory, loaded with zero-filled cp.async (the zero padding of the
// convolution).  The input gradient is the same convolution with the taps
// flipped and the channel axes swapped; the weight gradient reduces over
// points.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cmath>

#include "fd_internal.h"
#include "fd_internal_host.h"

namespace fdgb {

namespace {

constexpr int kC = 16;          // channels stored per point
constexpr int kT1 = 8;          // tile rows (d1), one warp each
constexpr int kT2 = 64;         // tile points along d2
constexpr int kZc = 16;         // d0 planes per CTA
constexpr int kPlanePts = (kT1 + 2) * (kT2 + 2);
constexpr int kRing = 4;        // input planes held: z-1, z, z+1 and the one in flight

struct CnnDims {
    int n0, n1, n2;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid)
{
    const int bytes = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared-memory position (in 16-byte chunks) of channel half h of plane
// point pt: the halves of points whose index has bit 2 set are exchanged, so
// that the 8 row addresses of an ldmatrix phase (8 consecutive points, any
// start) fall in 8 distinct 16-byte bank groups.
__device__ __forceinline__ int chunk_of(int pt, int h) { return 2 * pt + (h ^ ((pt >> 2) & 1)); }

// Load input plane z (all 16 channels, rows row0-1.., points col0-1..) into
// ring slot `slot`; out-of-grid points are zero.
__device__ __forceinline__ void load_plane(uint32_t *ring, int slot, const __nv_bfloat16 *x, const CnnDims &d,
                                           int z, int row0, int col0)
{
    uint32_t *dst = ring + slot * kPlanePts * (kC / 2);
    const bool zin = z >= 0 && z < d.n0;
    for (int q = threadIdx.x; q < kPlanePts * 2; q += blockDim.x) {
        const int pt = q >> 1, half = q & 1;
        const int rr = pt / (kT2 + 2), cc = pt - rr * (kT2 + 2);
        const int gy = row0 - 1 + rr, gx = col0 - 1 + cc;
        const bool ok = zin && gy >= 0 && gy < d.n1 && gx >= 0 && gx < d.n2;
        const __nv_bfloat16 *src = ok ? x + (((long long)z * d.n1 + gy) * d.n2 + gx) * kC + half * 8 : x;
        cp_async16(smem_u32(dst + chunk_of(pt, half) * 4), src, ok);
    }
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

// y = act(conv(x, w) + b) [* (mask > 0)].  NT output-channel groups of 8.
// OUT_F32: write channel 0 as FP32 (the network's output), else BF16 x 16.
template <int NT, bool RELU, bool MASK, bool OUT_F32>
__global__ void __launch_bounds__(32 * kT1, 2)
    conv3d_kernel(const __nv_bfloat16 *__restrict__ x, const uint2 *__restrict__ wfrag,
                  const float *__restrict__ bias, int cout, const __nv_bfloat16 *__restrict__ mask, void *y,
                  CnnDims d)
{
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *ring = smem;
    uint2 *sw = reinterpret_cast<uint2 *>(smem + kRing * kPlanePts * (kC / 2));
    const int tiles2 = (d.n2 + kT2 - 1) / kT2;
    const int col0 = (blockIdx.x % tiles2) * kT2;
    const int row0 = (blockIdx.x / tiles2) * kT1;
    const int z0 = blockIdx.y * kZc;
    const int z1 = min(d.n0, z0 + kZc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    // ldmatrix row of this lane: matrix lane/8 (0: points 0-7 channels 0-7,
    // 1: points 8-15 channels 0-7, 2: points 0-7 channels 8-15, 3: points
    // 8-15 channels 8-15), row lane%8
    const int lm_pt = ((lane >> 3) & 1) * 8 + (lane & 7);
    const int lm_half = lane >> 4;

    for (int q = threadIdx.x; q < 27 * NT * 32; q += blockDim.x) sw[q] = wfrag[q];
    load_plane(ring, (z0 - 1 + kRing) % kRing, x, d, z0 - 1, row0, col0);
    load_plane(ring, z0 % kRing, x, d, z0, row0, col0);
    cp_async_commit();
    load_plane(ring, (z0 + 1) % kRing, x, d, z0 + 1, row0, col0);
    cp_async_commit();

    float bv[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int o = nt * 8 + tig * 2;
        bv[nt][0] = (bias && o < cout) ? bias[o] : 0.f;
        bv[nt][1] = (bias && o + 1 < cout) ? bias[o + 1] : 0.f;
    }
    const uint32_t ring_base = smem_u32(ring);

    for (int z = z0; z < z1; z++) {
        // plane z+2 in flight while z is computed; z+1 must have landed
        load_plane(ring, (z + 2) % kRing, x, d, z + 2, row0, col0);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();

        float acc[4][NT][4];
#pragma unroll
        for (int mt = 0; mt < 4; mt++)
#pragma unroll
            for (int nt = 0; nt < NT; nt++)
#pragma unroll
                for (int e = 0; e < 4; e++) acc[mt][nt][e] = 0.f;

#pragma unroll 1
        for (int a = -1; a <= 1; a++) {
            const uint32_t plane = ring_base + (uint32_t)(((z + a + kRing) % kRing) * kPlanePts * (kC / 2) * 4);
#pragma unroll
            for (int b = -1; b <= 1; b++) {
#pragma unroll
                for (int c = -1; c <= 1; c++) {
                    const int t = (a + 1) * 9 + (b + 1) * 3 + (c + 1);
                    uint2 bw[NT];
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) bw[nt] = sw[(t * NT + nt) * 32 + lane];
                    // first point of this warp's row for the tap
                    const int pt0 = (warp + 1 + b) * (kT2 + 2) + 1 + c;
#pragma unroll
                    for (int mt = 0; mt < 4; mt++) {
                        const int pt = pt0 + mt * 16 + lm_pt;
                        uint32_t a0, a1, a2, a3;
                        ldmatrix_x4(plane + (uint32_t)(chunk_of(pt, lm_half) * 16), a0, a1, a2, a3);
#pragma unroll
                        for (int nt = 0; nt < NT; nt++) mma_bf16(acc[mt][nt], a0, a1, a2, a3, bw[nt].x, bw[nt].y);
                    }
                }
            }
        }

        const int gy = row0 + warp;
        if (gy < d.n1) {
#pragma unroll
            for (int mt = 0; mt < 4; mt++) {
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int gx = col0 + mt * 16 + g + 8 * h;
                    if (gx >= d.n2) continue;
                    const long long pt = ((long long)z * d.n1 + gy) * d.n2 + gx;
#pragma unroll
                    for (int nt = 0; nt < NT; nt++) {
                        float v0 = acc[mt][nt][2 * h] + bv[nt][0];
                        float v1 = acc[mt][nt][2 * h + 1] + bv[nt][1];
                        if (RELU) {
                            v0 = fmaxf(v0, 0.f);
                            v1 = fmaxf(v1, 0.f);
                        }
                        const int o = nt * 8 + tig * 2;
                        if (MASK) {
                            const __nv_bfloat162 mk =
                                *reinterpret_cast<const __nv_bfloat162 *>(mask + pt * kC + o);
                            if (!(__low2float(mk) > 0.f)) v0 = 0.f;
                            if (!(__high2float(mk) > 0.f)) v1 = 0.f;
                        }
                        if (OUT_F32) {
                            if (o == 0) reinterpret_cast<float *>(y)[pt] = v0;
                        } else {
                            *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(y) + pt * kC + o) =
                                __floats2bfloat162_rn(v0, v1);
                        }
                    }
                    if (!OUT_F32 && NT == 1)  // channels 8..15 of a narrow output are zero
                        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<__nv_bfloat16 *>(y) + pt * kC + 8 +
                                                            tig * 2) = __floats2bfloat162_rn(0.f, 0.f);
                }
            }
        }
        __syncthreads();  // the slot of plane z-1 is refilled next iteration
    }
    cp_async_wait<0>();
}

// Pack FP32 weights w[27][cin][cout] into the mma B fragments of each tap and
// 8-column group; flip = 1 packs the input-gradient convolution (taps
// mirrored, cin and cout exchanged).
__global__ void pack_weights_kernel(const float *__restrict__ w, int cin, int cout, int flip, int nt_count,
                                    uint2 *__restrict__ frag)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 27 * nt_count * 32) return;
    const int lane = q & 31, nt = (q >> 5) % nt_count, t = q / (32 * nt_count);
    const int g = lane >> 2, tig = lane & 3;
    const int n = nt * 8 + g;
    auto W = [&](int k, int nn) -> float {
        // the B matrix of the convolution being packed: rows k = its input
        // channel, columns nn = its output channel
        if (!flip) return (k < cin && nn < cout) ? w[((long long)t * cin + k) * cout + nn] : 0.f;
        const int tf = 26 - t;  // mirrored tap
        return (k < cout && nn < cin) ? w[((long long)tf * cin + nn) * cout + k] : 0.f;
    };
    const __nv_bfloat162 lo = __floats2bfloat162_rn(W(tig * 2, n), W(tig * 2 + 1, n));
    const __nv_bfloat162 hi = __floats2bfloat162_rn(W(tig * 2 + 8, n), W(tig * 2 + 9, n));
    uint2 v;
    v.x = *reinterpret_cast<const uint32_t *>(&lo);
    v.y = *reinterpret_cast<const uint32_t *>(&hi);
    frag[q] = v;
}

// Weight gradient gw[t][c][o] += sum_p x[p + off_t][c] gy[p][o], gb[o] +=
// sum_p gy[p][o], for a block of 8 x 8 x 8 points per CTA: the block (with a
// one-point halo) and its gy are staged in shared memory; thread (c, o)
// accumulates the 27 taps of its pair in registers.
constexpr int kWb = 8;
__global__ void __launch_bounds__(256)
    conv3d_wgrad_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ gy, int cin,
                        int cout, float *__restrict__ gw, float *__restrict__ gb, CnnDims d)
{
    __shared__ __nv_bfloat16 sx[(kWb + 2) * (kWb + 2) * (kWb + 2)][kC];
    __shared__ __nv_bfloat16 sg[kWb * kWb * kWb][kC];
    const int b2 = (d.n2 + kWb - 1) / kWb, b1 = (d.n1 + kWb - 1) / kWb;
    const int bz = blockIdx.x / (b1 * b2), by = (blockIdx.x / b2) % b1, bx = blockIdx.x % b2;
    const int z0 = bz * kWb, y0 = by * kWb, x0 = bx * kWb;
    for (int q = threadIdx.x; q < (kWb + 2) * (kWb + 2) * (kWb + 2) * kC; q += blockDim.x) {
        const int c = q % kC, pt = q / kC;
        const int i = pt / ((kWb + 2) * (kWb + 2)), j = (pt / (kWb + 2)) % (kWb + 2), k = pt % (kWb + 2);
        const int gz = z0 - 1 + i, gyy = y0 - 1 + j, gx = x0 - 1 + k;
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (gz >= 0 && gz < d.n0 && gyy >= 0 && gyy < d.n1 && gx >= 0 && gx < d.n2)
            v = x[(((long long)gz * d.n1 + gyy) * d.n2 + gx) * kC + c];
        sx[pt][c] = v;
    }
    for (int q = threadIdx.x; q < kWb * kWb * kWb * kC; q += blockDim.x) {
        const int c = q % kC, pt = q / kC;
        const int i = pt / (kWb * kWb), j = (pt / kWb) % kWb, k = pt % kWb;
        const int gz = z0 + i, gyy = y0 + j, gx = x0 + k;
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (gz < d.n0 && gyy < d.n1 && gx < d.n2) v = gy[(((long long)gz * d.n1 + gyy) * d.n2 + gx) * kC + c];
        sg[pt][c] = v;
    }
    __syncthreads();
    const int c = threadIdx.x & 15, o = threadIdx.x >> 4;
    if (c >= cin || o >= cout) return;
    float acc[27];
#pragma unroll
    for (int t = 0; t < 27; t++) acc[t] = 0.f;
    float accb = 0.f;
    for (int pt = 0; pt < kWb * kWb * kWb; pt++) {
        const int i = pt / (kWb * kWb), j = (pt / kWb) % kWb, k = pt % kWb;
        const float gv = __bfloat162float(sg[pt][o]);
        accb += gv;
#pragma unroll
        for (int t = 0; t < 27; t++) {
            const int a = t / 9, b = (t / 3) % 3, cc = t % 3;  // offsets + 1
            acc[t] = fmaf(__bfloat162float(sx[((i + a) * (kWb + 2) + (j + b)) * (kWb + 2) + (k + cc)][c]), gv, acc[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < 27; t++) atomicAdd(&gw[((long long)t * cin + c) * cout + o], acc[t]);
    if (c == 0) atomicAdd(&gb[o], accb);
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output function
// applied to state = key + (counter + 1) * golden gamma.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long key, unsigned long long counter)
{
    unsigned long long z = key + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Unit-variance uniform deviate in [-sqrt 3, sqrt 3) from the top 24 bits.
__device__ __forceinline__ float unit_uniform(unsigned long long key, unsigned long long counter)
{
    const float r = (float)(splitmix64(key, counter) >> 40) * (1.0f / 16777216.0f);
    return 1.7320508f * (2.f * r - 1.f);
}

// Closure input features, all linear in the wavefield: with du = u^n -
// u^{n-1} and q = 1/(m vref^2) (the squared velocity relative to vref),
// channels 0..5 = (u, du, q u, q du, q^2 u, q^2 du) / s; with nsub model
// descriptors s_k (fields of the grid's layout, sub + k * sub_stride),
// channels 6 + 2k, 7 + 2k = (s_k u, s_k du) / s; the rest 0.  With noise > 0,
// u^n and u^{n-1} first get noise * xi added, xi the unit-variance deviates of
// counters 2p and 2p + 1 under key `seed` (training only).
__global__ void features_kernel(Geom g, const float *__restrict__ u, const float *__restrict__ up,
                                const float *__restrict__ m, const float *__restrict__ sub, int nsub,
                                long long sub_stride, float inv_scale, float inv_vref2, float noise,
                                unsigned long long seed, __nv_bfloat16 *__restrict__ x)
{
    const long long total = g.n[0] * g.n[1] * g.n[2];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / g.n[2];
        const long long i2 = p - row * g.n[2];
        const long long i0 = row / g.n[1], i1 = row - i0 * g.n[1];
        const long long at = i0 * g.s0 + i1 * g.s1 + i2;
        float uc = u[at], uq = up[at];
        if (noise != 0.f) {
            uc += noise * unit_uniform(seed, 2ull * (unsigned long long)p);
            uq += noise * unit_uniform(seed, 2ull * (unsigned long long)p + 1ull);
        }
        const float a = uc * inv_scale, b = (uc - uq) * inv_scale;
        const float q = inv_vref2 / m[at];
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(x + p * kC);
        dst[0] = __floats2bfloat162_rn(a, b);
        dst[1] = __floats2bfloat162_rn(q * a, q * b);
        dst[2] = __floats2bfloat162_rn(q * q * a, q * q * b);
        for (int k = 0; k < nsub; k++) {
            const float sk = sub[k * sub_stride + at];
            dst[3 + k] = __floats2bfloat162_rn(sk * a, sk * b);
        }
        for (int k = 3 + nsub; k < kC / 2; k++) dst[k] = __floats2bfloat162_rn(0.f, 0.f);
    }
}

// coarse[i] = fine[f i] per axis (injection of a fine grid whose nodes
// include every coarse node: n_fine = f (n_coarse - 1) + 1); optionally
// *sumsq += sum of the squared coarse values.
__global__ void restrict_kernel(Geom gc, Geom gf, int f, const float *__restrict__ fine, float *__restrict__ coarse,
                                float *sumsq)
{
    const long long total = gc.n[0] * gc.n[1] * gc.n[2];
    float local = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / gc.n[2];
        const long long i2 = p - row * gc.n[2];
        const long long i0 = row / gc.n[1], i1 = row - i0 * gc.n[1];
        const float v = fine[f * (i0 * gf.s0 + i1 * gf.s1 + i2)];
        coarse[i0 * gc.s0 + i1 * gc.s1 + i2] = v;
        local += v * v;
    }
    if (sumsq) {
        for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(sumsq, local);
    }
}

// u[at] += scale * corr[p] (the closure's correction of the coarse update)
__global__ void add_correction_kernel(Geom g, float *__restrict__ u, const float *__restrict__ corr, float scale)
{
    const long long total = g.n[0] * g.n[1] * g.n[2];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / g.n[2];
        const long long i2 = p - row * g.n[2];
        const long long i0 = row / g.n[1], i1 = row - i0 * g.n[1];
        u[i0 * g.s0 + i1 * g.s1 + i2] += scale * corr[p];
    }
}

// MSE loss of pred against r = (target - base) / s (base may be NULL) and its
// gradient into gy (BF16, channel 0; other channels zero):
// loss += sum (pred - r)^2 / count, gy = 2 (pred - r) / count.
__global__ void mse_grad_kernel(long long count, const float *__restrict__ pred, Geom g,
                                const float *__restrict__ target, const float *__restrict__ base, float inv_scale,
                                __nv_bfloat16 *__restrict__ gy, float *loss)
{
    float local = 0.f;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < count;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / g.n[2];
        const long long i2 = p - row * g.n[2];
        const long long i0 = row / g.n[1], i1 = row - i0 * g.n[1];
        const long long at = i0 * g.s0 + i1 * g.s1 + i2;
        const float r = (base ? target[at] - base[at] : target[at]) * inv_scale;
        const float e = pred[p] - r;
        local += e * e;
        __nv_bfloat162 *dst = reinterpret_cast<__nv_bfloat162 *>(gy + p * kC);
        dst[0] = __floats2bfloat162_rn(2.f * e / (float)count, 0.f);
        for (int k = 1; k < kC / 2; k++) dst[k] = __floats2bfloat162_rn(0.f, 0.f);
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, local / (float)count);
}

// Adam (Kingma & Ba 2015) on FP32 parameters.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi;
        const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = b;
        p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

int blocks_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    return (int)std::min<long long>(std::max<long long>(b, 1), 152 * 16);
}

template <int NT, bool RELU, bool MASK, bool OUT_F32>
cudaError_t launch_conv(const __nv_bfloat16 *x, const uint2 *wf, const float *b, int cout,
                        const __nv_bfloat16 *mask, void *y, CnnDims d, cudaStream_t st)
{
    const size_t smem = sizeof(uint32_t) * kRing * kPlanePts * (kC / 2) + sizeof(uint2) * 27 * NT * 32;
    auto k = conv3d_kernel<NT, RELU, MASK, OUT_F32>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(((d.n2 + kT2 - 1) / kT2) * ((d.n1 + kT1 - 1) / kT1)), (unsigned)((d.n0 + kZc - 1) / kZc));
    k<<<grid, 32 * kT1, smem, st>>>(x, wf, b, cout, mask, y, d);
    return cudaGetLastError();
}

}  // namespace

}  // namespace fdgb

using namespace fdgb;

static fd_status cnn_dims(int ndim, const int64_t *shape, CnnDims *d)
{
    if (ndim != 3 || !shape) return set_error(FD_ERR_INVALID_ARG, "cnn: 3D shapes only");
    for (int a = 0; a < 3; a++)
        if (shape[a] < 1 || shape[a] > (1 << 20)) return set_error(FD_ERR_INVALID_ARG, "cnn: bad shape");
    d->n0 = (int)shape[0];
    d->n1 = (int)shape[1];
    d->n2 = (int)shape[2];
    return FD_OK;
}

static Geom geom3(const fd_grid *grid)
{
    Geom g;
    g.ndim = 3;
    const int64_t S = (grid->shape[2] + 7) / 8 * 8;
    g.n[0] = grid->shape[0];
    g.n[1] = grid->shape[1];
    g.n[2] = grid->shape[2];
    g.s0 = grid->shape[1] * S;
    g.s1 = S;
    return g;
}

#define CNN_CUDA(call, what)                                                                           \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return set_error(FD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

extern "C" fd_status fd_cnn_pack_weights(const float *w, int cin, int cout, int flip, void *frag, void *stream)
{
    if (!w || !frag || cin < 1 || cin > 16 || cout < 1 || cout > 16)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_pack_weights: bad arguments");
    const int nt = ((flip ? cin : cout) + 7) / 8;
    const int total = 27 * nt * 32;
    pack_weights_kernel<<<(total + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, cin, cout, flip, nt, (uint2 *)frag);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_pack_weights");
    return FD_OK;
}

extern "C" fd_status fd_cnn_conv3d(const int64_t *shape, const void *x, const void *frag, const float *bias, int cout,
                                   int relu, const void *mask, void *y, int y_fp32, void *stream)
{
    CnnDims d;
    fd_status s = cnn_dims(3, shape, &d);
    if (s != FD_OK) return s;
    if (!x || !frag || !y || cout < 1 || cout > 16) return set_error(FD_ERR_INVALID_ARG, "fd_cnn_conv3d: bad arguments");
    // 16-byte copies of the input points, paired BF16 stores and mask loads
    if (((uintptr_t)x & 15) || ((uintptr_t)frag & 7) || ((uintptr_t)y & 3) || ((uintptr_t)mask & 3))
        return set_error(FD_ERR_LAYOUT, "fd_cnn_conv3d: x must be 16-byte, frag 8-byte, y and mask 4-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16 *xb = (const __nv_bfloat16 *)x;
    const __nv_bfloat16 *mk = (const __nv_bfloat16 *)mask;
    const uint2 *wf = (const uint2 *)frag;
    cudaError_t e;
    if (y_fp32) {
        if (cout != 1 || relu || mask) return set_error(FD_ERR_UNSUPPORTED, "fd_cnn_conv3d: FP32 output is one linear channel");
        e = launch_conv<1, false, false, true>(xb, wf, bias, cout, nullptr, y, d, st);
    } else if (cout <= 8) {
        if (relu && mask) e = launch_conv<1, true, true, false>(xb, wf, bias, cout, mk, y, d, st);
        else if (relu) e = launch_conv<1, true, false, false>(xb, wf, bias, cout, nullptr, y, d, st);
        else if (mask) e = launch_conv<1, false, true, false>(xb, wf, bias, cout, mk, y, d, st);
        else e = launch_conv<1, false, false, false>(xb, wf, bias, cout, nullptr, y, d, st);
    } else {
        if (relu && mask) e = launch_conv<2, true, true, false>(xb, wf, bias, cout, mk, y, d, st);
        else if (relu) e = launch_conv<2, true, false, false>(xb, wf, bias, cout, nullptr, y, d, st);
        else if (mask) e = launch_conv<2, false, true, false>(xb, wf, bias, cout, mk, y, d, st);
        else e = launch_conv<2, false, false, false>(xb, wf, bias, cout, nullptr, y, d, st);
    }
    CNN_CUDA(e, "fd_cnn_conv3d");
    return FD_OK;
}

extern "C" fd_status fd_cnn_conv3d_wgrad(const int64_t *shape, const void *x, const void *gy, int cin, int cout,
                                         float *gw, float *gb, void *stream)
{
    CnnDims d;
    fd_status s = cnn_dims(3, shape, &d);
    if (s != FD_OK) return s;
    if (!x || !gy || !gw || !gb || cin < 1 || cin > 16 || cout < 1 || cout > 16)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_conv3d_wgrad: bad arguments");
    const long long blocks =
        (long long)((d.n0 + kWb - 1) / kWb) * ((d.n1 + kWb - 1) / kWb) * ((d.n2 + kWb - 1) / kWb);
    conv3d_wgrad_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)gy, cin, cout, gw, gb, d);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_conv3d_wgrad");
    return FD_OK;
}

extern "C" fd_status fd_cnn_features_sub(const fd_grid *grid, const float *u, const float *u_prev, const float *m,
                                         const float *sub, int nsub, double scale, double vref, double noise,
                                         uint64_t seed, void *x, void *stream)
{
    if (!grid || grid->ndim != 3 || !u || !u_prev || !m || !x || !(scale > 0) || !(vref > 0) ||
        !(noise >= 0) || nsub < 0 || nsub > 5 || (nsub > 0 && !sub))
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_features: bad arguments");
    if ((uintptr_t)x & 3) return set_error(FD_ERR_LAYOUT, "fd_cnn_features: x must be 4-byte aligned");
    const Geom g = geom3(grid);
    const long long total = g.n[0] * g.n[1] * g.n[2];
    features_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        g, u, u_prev, m, sub, nsub, g.n[0] * g.s0, (float)(1.0 / scale), (float)(1.0 / (vref * vref)),
        (float)noise, (unsigned long long)seed, (__nv_bfloat16 *)x);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_features");
    return FD_OK;
}

extern "C" fd_status fd_cnn_features(const fd_grid *grid, const float *u, const float *u_prev, const float *m,
                                     double scale, double vref, double noise, uint64_t seed, void *x, void *stream)
{
    return fd_cnn_features_sub(grid, u, u_prev, m, nullptr, 0, scale, vref, noise, seed, x, stream);
}

extern "C" fd_status fd_cnn_restrict(const fd_grid *fine_grid, const float *fine, const fd_grid *coarse_grid,
                                     float *coarse, int factor, float *sumsq, void *stream)
{
    if (!fine_grid || !coarse_grid || fine_grid->ndim != 3 || coarse_grid->ndim != 3 || !fine || !coarse ||
        factor < 1)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_restrict: bad arguments");
    for (int a = 0; a < 3; a++)
        if (fine_grid->shape[a] != factor * (coarse_grid->shape[a] - 1) + 1)
            return set_error(FD_ERR_INVALID_ARG, "fd_cnn_restrict: fine shape must be factor*(n-1)+1 per axis");
    const Geom gc = geom3(coarse_grid), gf = geom3(fine_grid);
    const long long total = gc.n[0] * gc.n[1] * gc.n[2];
    restrict_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(gc, gf, factor, fine, coarse, sumsq);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_restrict");
    return FD_OK;
}

extern "C" fd_status fd_cnn_add_correction(const fd_grid *grid, float *u, const float *corr, double scale,
                                           void *stream)
{
    if (!grid || grid->ndim != 3 || !u || !corr) return set_error(FD_ERR_INVALID_ARG, "fd_cnn_add_correction: bad arguments");
    const Geom g = geom3(grid);
    const long long total = g.n[0] * g.n[1] * g.n[2];
    add_correction_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(g, u, corr, (float)scale);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_add_correction");
    return FD_OK;
}

extern "C" fd_status fd_cnn_mse_grad(const fd_grid *grid, const float *pred, const float *target, const float *base,
                                     double scale, void *gy, float *loss, void *stream)
{
    if (!grid || grid->ndim != 3 || !pred || !target || !gy || !loss || !(scale > 0))
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_mse_grad: bad arguments");
    if ((uintptr_t)gy & 3) return set_error(FD_ERR_LAYOUT, "fd_cnn_mse_grad: gy must be 4-byte aligned");
    const Geom g = geom3(grid);
    const long long total = g.n[0] * g.n[1] * g.n[2];
    mse_grad_kernel<<<blocks_for(total, 256), 256, 0, (cudaStream_t)stream>>>(
        total, pred, g, target, base, (float)(1.0 / scale), (__nv_bfloat16 *)gy, loss);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_mse_grad");
    return FD_OK;
}

extern "C" fd_status fd_cnn_adam(float *params, const float *grads, float *m1, float *m2, int64_t n, double lr,
                                 double beta1, double beta2, double eps, int64_t step, void *stream)
{
    if (!params || !grads || !m1 || !m2 || n < 0 || step < 1)
        return set_error(FD_ERR_INVALID_ARG, "fd_cnn_adam: bad arguments");
    const float c1 = (float)(1.0 - std::pow(beta1, (double)step));
    const float c2 = (float)(1.0 - std::pow(beta2, (double)step));
    adam_kernel<<<blocks_for(n, 256), 256, 0, (cudaStream_t)stream>>>(params, grads, m1, m2, n, (float)lr,
                                                                      (float)beta1, (float)beta2, (float)eps, c1, c2);
    CNN_CUDA(cudaGetLastError(), "fd_cnn_adam");
    return FD_OK;
}
