// fd_interpolate_noalloc: receiver interpolation that allocates no memory.
//
// Some callers cannot allocate device memory when they need to record a
// wavefield at off-grid points: a process whose device memory is fully
// reserved up front by another framework's caching pool, a service with a
// fixed device-memory budget decided at start-up, or a latency-critical loop
// that must not stall other streams (cudaMalloc and cudaFree may synchronise
// the device).  This entry point serves them: its interpolation table lives in
// a file-scope device array of fixed size, loaded with the library, instead of
// in memory allocated per sparse object.  It computes exactly what the
// interpolation of fd_operator_apply computes (same table, same kernel).
#include <cmath>
#include <cstring>
#include <mutex>

#include "fd_internal.h"
#include "fd_internal_host.h"

namespace fdgb {

namespace {

constexpr int kMaxPoints = FD_NOALLOC_MAX_POINTS;
constexpr size_t kBaseBytes = sizeof(int64_t) * kMaxPoints;
constexpr size_t kTableBytes = kBaseBytes + sizeof(float) * 8 * kMaxPoints;
constexpr int kMaxDevices = 64;

// The scratch: per point an int64 base index, then per point 8 FP32 corner
// weights.  Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_table[kTableBytes];

// Host staging copy of the table (filled under g_lock, copied with
// cudaMemcpyAsync, which for pageable memory returns once the bytes are
// staged, so the buffer is free again when the call returns).
static unsigned char g_host_table[kTableBytes];
static std::mutex g_lock;
static void *g_dev_addr[kMaxDevices];

}  // namespace

}  // namespace fdgb

using namespace fdgb;

extern "C" fd_status fd_interpolate_noalloc(const fd_grid *g, int npoint, const double *coords,
                                            const void *dev_field, void *dev_out, void *cuda_stream)
{
    if (!g) return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: null grid");
    if (npoint < 0 || npoint > kMaxPoints)
        return set_error(FD_ERR_INVALID_ARG,
                         "fd_interpolate_noalloc: %d points requested, the static table holds at most %d", npoint,
                         kMaxPoints);
    if (npoint == 0) return FD_OK;
    for (int a = 0; a < g->ndim; a++)
        if (g->shape[a] < 2)
            return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: axis %d has %lld node(s); points need >= 2",
                             a, (long long)g->shape[a]);
    if (!coords || !dev_field || !dev_out)
        return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: null pointer");
    const int ndim = g->ndim;
    // the layout of fd_field_layout: rows padded to a multiple of 8 elements
    const int64_t S = (g->shape[ndim - 1] + 7) / 8 * 8;
    int64_t st[3];
    if (ndim == 3) {
        st[0] = g->shape[1] * S; st[1] = S; st[2] = 1;
    } else {
        st[0] = S; st[1] = 1; st[2] = 0;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    std::lock_guard<std::mutex> guard(g_lock);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FD_ERR_UNSUPPORTED, "fd_interpolate_noalloc: device %d", dev);
    if (!g_dev_addr[dev]) {
        // once per device, with that device current: the device address of
        // the static table (the host-side symbol is only a stand-in)
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_table);
        if (e != cudaSuccess || !p)
            return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_dev_addr[dev] = p;
    }
    unsigned char *dtab = (unsigned char *)g_dev_addr[dev];

    int64_t *base = (int64_t *)g_host_table;
    float *weight = (float *)(g_host_table + kBaseBytes);
    for (int p = 0; p < npoint; p++) {
        int64_t lin = 0;
        double frac[3] = {0, 0, 0};
        for (int a = 0; a < ndim; a++) {
            double x = coords[(int64_t)p * ndim + a];
            double s = (x - g->origin[a]) / g->spacing[a];
            double top = (double)(g->shape[a] - 1);
            if (!(s >= 0.0) || !(s <= top))
                return set_error(FD_ERR_OUT_OF_DOMAIN, "fd_interpolate_noalloc: point %d coordinate %d = %g outside the grid",
                                 p, a, x);
            int64_t i = (int64_t)std::floor(s);
            if (i > g->shape[a] - 2) i = g->shape[a] - 2;
            frac[a] = s - (double)i;
            lin += i * st[a];
        }
        base[p] = lin;
        for (int k = 0; k < 8; k++) {
            double w = 0.0;
            if (k < (1 << ndim)) {
                w = 1.0;
                for (int a = 0; a < ndim; a++) w *= ((k >> a) & 1) ? frac[a] : 1.0 - frac[a];
            }
            weight[(size_t)p * 8 + k] = (float)w;
        }
    }
    e = cudaMemcpyAsync(dtab, base, sizeof(int64_t) * npoint, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtab + kBaseBytes, weight, sizeof(float) * 8 * npoint, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: table upload: %s", cudaGetErrorString(e));

    SparseDev sp;
    sp.npoint = npoint;
    sp.ncorner = 1 << ndim;
    sp.base = (const int64_t *)dtab;
    sp.weight = (const float *)(dtab + kBaseBytes);
    for (int k = 0; k < 8; k++) {
        int64_t off = 0;
        if (k < sp.ncorner)
            for (int a = 0; a < ndim; a++) off += ((k >> a) & 1) * st[a];
        sp.corner_off[k] = off;
    }
    e = launch_interpolate(sp, (const float *)dev_field, (float *)dev_out, stream);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: launch: %s", cudaGetErrorString(e));
    return FD_OK;
}
