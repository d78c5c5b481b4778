// fd_interpolate_noalloc: receiver interpolation that allocates no memory.
//
// Some callers cannot allocate device memory when they need to record a
// wavefield at off-grid points: a process whose device memory is fully
// reserved up front by another framework's caching pool, a service with a
// fixed device-memory budget decided at start-up, or a latency-critical loop
// that must not stall other streams (cudaMalloc and cudaFree may synchronise
// the device).  This entry point serves them: its interpolation table lives in
// a file-scope device array of fixed size instead of in memory allocated per
// sparse object.  It computes exactly what the interpolation of
// fd_operator_apply computes: the same table builder (linear_table) and the
// same kernel.
//
// The array belongs to this file's module, which CUDA loads lazily: on each
// device the array is allocated when the module is first used there, i.e. at
// the first call of this entry point on that device.  A call with no points
// does only that set-up (it also loads the interpolation kernel), so a caller
// can pay for it at start-up, while memory can still be had and before any
// stream capture; after it, calls on that device allocate nothing.
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

// Host staging copy of the table, filled under g_lock and copied with
// cudaMemcpyAsync.  From pageable memory that copy first waits for the
// stream's earlier work and returns once the bytes are staged, so the buffer
// is free again when the call returns.
static unsigned char g_host_table[kTableBytes];
static std::mutex g_lock;
static void *g_dev_addr[kMaxDevices];

}  // namespace

}  // namespace fdgb

using namespace fdgb;

// Once per device, with that device current: the device address of the
// static table (in host code the symbol is only a stand-in), and the
// interpolation kernel's module loaded.  Called under g_lock.
static fd_status noalloc_setup(unsigned char **dtab)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FD_ERR_UNSUPPORTED, "fd_interpolate_noalloc: device %d", dev);
    if (!g_dev_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_table);
        if (e != cudaSuccess || !p)
            return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        e = prepare_interpolate();
        if (e != cudaSuccess)
            return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: loading the interpolation kernel: %s",
                             cudaGetErrorString(e));
        g_dev_addr[dev] = p;
    }
    *dtab = (unsigned char *)g_dev_addr[dev];
    return FD_OK;
}

extern "C" fd_status fd_interpolate_noalloc(const fd_grid *g, int npoint, const double *coords,
                                            const void *dev_field, void *dev_out, void *cuda_stream)
{
    if (npoint < 0 || npoint > kMaxPoints)
        return set_error(FD_ERR_INVALID_ARG,
                         "fd_interpolate_noalloc: %d points requested, the static table holds at most %d", npoint,
                         kMaxPoints);
    std::lock_guard<std::mutex> guard(g_lock);
    unsigned char *dtab = nullptr;
    fd_status st = noalloc_setup(&dtab);
    if (st != FD_OK || npoint == 0) return st;

    if (!g) return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: null grid");
    for (int a = 0; a < g->ndim; a++)
        if (g->shape[a] < 2)
            return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: axis %d has %lld node(s); points need >= 2",
                             a, (long long)g->shape[a]);
    if (!coords || !dev_field || !dev_out)
        return set_error(FD_ERR_INVALID_ARG, "fd_interpolate_noalloc: null pointer");
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    int64_t *base = (int64_t *)g_host_table;
    float *weight = (float *)(g_host_table + kBaseBytes);
    st = linear_table(*g, npoint, coords, base, weight, "fd_interpolate_noalloc");
    if (st != FD_OK) return st;
    cudaError_t e = cudaMemcpyAsync(dtab, base, sizeof(int64_t) * npoint, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtab + kBaseBytes, weight, sizeof(float) * 8 * npoint, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: table upload: %s", cudaGetErrorString(e));

    SparseDev sp;
    sp.npoint = npoint;
    sp.ncorner = 1 << g->ndim;
    sp.base = (const int64_t *)dtab;
    sp.weight = (const float *)(dtab + kBaseBytes);
    corner_offsets(*g, sp.corner_off);
    e = launch_interpolate(sp, (const float *)dev_field, (float *)dev_out, stream);
    if (e != cudaSuccess) return set_error(FD_ERR_CUDA, "fd_interpolate_noalloc: launch: %s", cudaGetErrorString(e));
    return FD_OK;
}
