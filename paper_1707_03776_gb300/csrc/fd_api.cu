// C-ABI of libfdgb: grids, fields, sparse points and operators (include/fd.h).
//
// Host logic only: validation, layouts, interpolation tables, the stability
// check and the per-step launch sequence.  All arithmetic on grid data runs
// in the kernel files.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fd_internal.h"
#include "fd_internal_host.h"
#include "fd_tma.h"

struct fd_field {
    fd_grid g;
    int levels;
    float *slot[2];
};

struct fd_sparse {
    fd_grid g;
    int npoint;
    int64_t *d_base;   // library-owned
    float *d_weight;   // library-owned, [npoint][8]
    float *trace;      // caller-owned, row n at trace + n * stride
    int64_t nt;
    int64_t stride;
    cudaStream_t alloc_stream;
    fdgb::SparseDev dev;
    std::vector<int64_t> h_base;   // host copy of the table (for the fused kernel's layout)
    std::vector<float> h_weight;
};

struct fd_operator {
    int kind;
    int so;
    fd_field *u, *m, *eta;
    double a;
    fd_sparse *src, *rec;
    cudaStream_t stream;
    unsigned flags;
    fdgb::Geom geom;
    fdgb::Coef coef;
    double lambda_max;     // max over theta of the Laplacian symbol (1/length^2)
    float *c, *d;          // acoustic coefficient fields (library-owned)
    int *status;           // device status word (library-owned)
    double coef_dt;        // dt the coefficient fields were computed for (<0: none)
    double m_min;          // min(m) over the grid
    int64_t launches;
    fdgb::TmaPlan tma;     // tiled-kernel plan (tensor maps, tiling)
    fdgb::PairPlan pair;   // two steps per sweep (3D acoustic, SO 4..8)
    int want_sweep;        // 3D acoustic steps per sweep: 0 planner, 1, 2
    fdgb::ClusterPlan cluster;  // small 2D grids: whole run in one cluster launch
    int want_k;            // forced steps per cluster exchange (0: planner)
    float jac_wr, jac_wc;  // Laplace: weights of the row and column neighbours
    void *conv_res;        // Laplace: device {int64 steps, double r, double sum}
    // stencil-kernel timing (fd_operator_profile)
    std::vector<cudaEvent_t> prof_ev;  // pairs: start, stop
    // receiver interpolation beside the grid update (tiled path): a side
    // stream and the two events that order it with the operator's stream
    cudaStream_t side;
    cudaEvent_t ev_u, ev_rec;
    int64_t prof_max;
    int64_t prof_used;
};

namespace fdgb {

static thread_local std::string g_last_error;

fd_status set_error(fd_status status, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

static fd_status cuda_error(cudaError_t e, const char *what)
{
    return set_error(FD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define FD_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return fdgb::cuda_error(e_, what); \
    } while (0)

static int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Row pitch (elements) of the contiguous axis.
int64_t row_pitch(const fd_grid &g) { return round_up(g.shape[g.ndim - 1], 8); }

void layout_of(const fd_grid &g, int64_t *padded, int64_t *strides)
{
    int64_t S = row_pitch(g);
    if (g.ndim == 3) {
        padded[0] = g.shape[0]; padded[1] = g.shape[1]; padded[2] = S;
        strides[0] = g.shape[1] * S; strides[1] = S; strides[2] = 1;
    } else {
        padded[0] = g.shape[0]; padded[1] = S;
        strides[0] = S; strides[1] = 1;
    }
}

// Linear offset of corner k (bit a of k: +1 along axis a) from a point's
// lowest corner, in the slot layout; corners past 2^ndim are 0.
void corner_offsets(const fd_grid &g, int64_t off[8])
{
    int64_t padded[3], st[3];
    layout_of(g, padded, st);
    for (int k = 0; k < 8; k++) {
        off[k] = 0;
        if (k < (1 << g.ndim))
            for (int a = 0; a < g.ndim; a++) off[k] += ((k >> a) & 1) * st[a];
    }
}

// The linear-interpolation table of the paper's PointData (the weights of
// `interpolate` and `inject`): per point the slot-layout index of its lowest
// corner and the 2^ndim products of (1 - f) or f per axis, with
// s = (x - origin)/h, i = floor(s) clamped to n - 2 (a point on the upper
// face takes weight 1 on the last node) and f = s - i, all in FP64 and each
// weight rounded once to FP32 (unused corners 0).  Points outside
// [origin, origin + (n-1) h] are rejected.
fd_status linear_table(const fd_grid &g, int npoint, const double *coords, int64_t *base, float *weight,
                       const char *who)
{
    const int ndim = g.ndim;
    int64_t padded[3], st[3];
    layout_of(g, padded, st);
    for (int p = 0; p < npoint; p++) {
        int64_t lin = 0;
        double frac[3] = {0, 0, 0};
        for (int a = 0; a < ndim; a++) {
            double x = coords[(int64_t)p * ndim + a];
            double s = (x - g.origin[a]) / g.spacing[a];
            double top = (double)(g.shape[a] - 1);
            if (!(s >= 0.0) || !(s <= top))
                return set_error(FD_ERR_OUT_OF_DOMAIN, "%s: point %d coordinate %d = %g outside [%g, %g]", who, p,
                                 a, x, g.origin[a], g.origin[a] + top * g.spacing[a]);
            int64_t i = (int64_t)std::floor(s);
            if (i > g.shape[a] - 2) i = g.shape[a] - 2;
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
    return FD_OK;
}

static int64_t slot_elems(const fd_grid &g)
{
    int64_t S = row_pitch(g);
    return g.ndim == 3 ? g.shape[0] * g.shape[1] * S : g.shape[0] * S;
}

static Geom geom_of(const fd_grid &g)
{
    Geom q;
    q.ndim = g.ndim;
    int64_t S = row_pitch(g);
    if (g.ndim == 3) {
        q.n[0] = g.shape[0]; q.n[1] = g.shape[1]; q.n[2] = g.shape[2];
        q.s0 = g.shape[1] * S; q.s1 = S;
    } else {
        q.n[0] = 1; q.n[1] = g.shape[0]; q.n[2] = g.shape[1];
        q.s0 = g.shape[0] * S; q.s1 = S;
    }
    return q;
}

static bool same_shape(const fd_grid &a, const fd_grid &b)
{
    if (a.ndim != b.ndim) return false;
    for (int i = 0; i < a.ndim; i++)
        if (a.shape[i] != b.shape[i]) return false;
    return true;
}

// Max over theta in [0, pi] of -(w0 + 2 sum_k w_k cos(k theta)): the largest
// eigenvalue magnitude of the 1D central stencil (in units of 1/h^2).
static double symbol_max(const double *w, int M)
{
    double best = 0.0;
    const int samples = 4096;
    for (int s = 0; s <= samples; s++) {
        double th = M_PI * s / samples;
        double v = w[0];
        for (int k = 1; k <= M; k++) v += 2.0 * w[k] * std::cos(k * th);
        if (-v > best) best = -v;
    }
    return best;
}

}  // namespace fdgb

using namespace fdgb;

// ---------------------------------------------------------------------------
// status and version
// ---------------------------------------------------------------------------

extern "C" const char *fd_status_string(fd_status s)
{
    switch (s) {
    case FD_OK: return "FD_OK";
    case FD_ERR_INVALID_ARG: return "FD_ERR_INVALID_ARG";
    case FD_ERR_UNSUPPORTED: return "FD_ERR_UNSUPPORTED";
    case FD_ERR_LAYOUT: return "FD_ERR_LAYOUT";
    case FD_ERR_OUT_OF_DOMAIN: return "FD_ERR_OUT_OF_DOMAIN";
    case FD_ERR_UNSTABLE: return "FD_ERR_UNSTABLE";
    case FD_ERR_CUDA: return "FD_ERR_CUDA";
    case FD_ERR_TIMEOUT: return "FD_ERR_TIMEOUT";
    case FD_ERR_NOMEM: return "FD_ERR_NOMEM";
    }
    return "FD_ERR_UNKNOWN";
}

extern "C" const char *fd_last_error(void) { return g_last_error.c_str(); }

extern "C" int fd_version(void) { return 100; }

// ---------------------------------------------------------------------------
// grid
// ---------------------------------------------------------------------------

extern "C" fd_status fd_grid_create(int ndim, const int64_t *shape, const double *spacing,
                                    const double *origin, fd_grid **out)
{
    if (!out || !shape || !spacing) return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: null pointer");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: ndim must be 2 or 3");
    fd_grid g;
    std::memset(&g, 0, sizeof g);
    g.ndim = ndim;
    for (int a = 0; a < ndim; a++) {
        if (shape[a] < 2 || shape[a] > (int64_t(1) << 24))
            return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: shape[%d] = %lld out of [2, 2^24]", a,
                             (long long)shape[a]);
        if (!(spacing[a] > 0.0) || !std::isfinite(spacing[a]))
            return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: spacing[%d] must be > 0", a);
        g.shape[a] = shape[a];
        g.spacing[a] = spacing[a];
        g.origin[a] = origin ? origin[a] : 0.0;
        if (!std::isfinite(g.origin[a])) return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: bad origin");
    }
    int64_t total = 1;
    for (int a = 0; a < ndim; a++) total *= shape[a];
    if (total > (int64_t(1) << 40)) return set_error(FD_ERR_INVALID_ARG, "fd_grid_create: grid too large");
    fd_grid *p = new (std::nothrow) fd_grid(g);
    if (!p) return set_error(FD_ERR_NOMEM, "fd_grid_create: out of host memory");
    *out = p;
    return FD_OK;
}

extern "C" void fd_grid_destroy(fd_grid *g) { delete g; }

// ---------------------------------------------------------------------------
// fields
// ---------------------------------------------------------------------------

extern "C" fd_status fd_field_layout(const fd_grid *g, int space_order, int64_t *padded_shape,
                                     int64_t *strides, int64_t *interior_offset)
{
    if (!g || !padded_shape || !strides) return set_error(FD_ERR_INVALID_ARG, "fd_field_layout: null pointer");
    if (space_order < 2 || space_order > 16 || space_order % 2)
        return set_error(FD_ERR_UNSUPPORTED, "fd_field_layout: space order must be even, 2..16");
    layout_of(*g, padded_shape, strides);
    if (interior_offset) *interior_offset = 0;
    return FD_OK;
}

extern "C" fd_status fd_field_wrap(const fd_grid *g, int levels, void *const *dev_ptrs,
                                   const int64_t *strides, fd_field **out)
{
    if (!g || !dev_ptrs || !out) return set_error(FD_ERR_INVALID_ARG, "fd_field_wrap: null pointer");
    *out = nullptr;
    if (levels != 1 && levels != 2) return set_error(FD_ERR_INVALID_ARG, "fd_field_wrap: levels must be 1 or 2");
    int64_t padded[3], st[3];
    layout_of(*g, padded, st);
    if (strides)
        for (int a = 0; a < g->ndim; a++)
            if (strides[a] != st[a])
                return set_error(FD_ERR_LAYOUT, "fd_field_wrap: stride[%d] = %lld, layout needs %lld", a,
                                 (long long)strides[a], (long long)st[a]);
    fd_field f;
    f.g = *g;
    f.levels = levels;
    f.slot[0] = f.slot[1] = nullptr;
    for (int l = 0; l < levels; l++) {
        if (!dev_ptrs[l]) return set_error(FD_ERR_INVALID_ARG, "fd_field_wrap: null slot %d", l);
        if (((uintptr_t)dev_ptrs[l]) % 32 != 0)
            return set_error(FD_ERR_LAYOUT, "fd_field_wrap: slot %d is not 32-byte aligned", l);
        f.slot[l] = (float *)dev_ptrs[l];
    }
    if (levels == 2 && f.slot[0] == f.slot[1])
        return set_error(FD_ERR_INVALID_ARG, "fd_field_wrap: the two slots alias");
    fd_field *p = new (std::nothrow) fd_field(f);
    if (!p) return set_error(FD_ERR_NOMEM, "fd_field_wrap: out of host memory");
    *out = p;
    return FD_OK;
}

extern "C" void fd_field_destroy(fd_field *f) { delete f; }

// ---------------------------------------------------------------------------
// sparse points
// ---------------------------------------------------------------------------

extern "C" fd_status fd_sparse_create(const fd_grid *g, int npoint, const double *coords,
                                      void *dev_trace, int64_t nt, int64_t trace_stride,
                                      void *cuda_stream, fd_sparse **out)
{
    if (!g || !out) return set_error(FD_ERR_INVALID_ARG, "fd_sparse_create: null pointer");
    *out = nullptr;
    if (npoint < 0) return set_error(FD_ERR_INVALID_ARG, "fd_sparse_create: npoint < 0");
    if (npoint > 0 && (!coords || !dev_trace))
        return set_error(FD_ERR_INVALID_ARG, "fd_sparse_create: null coordinates or trace");
    if (nt < 0 || (npoint > 0 && trace_stride < npoint))
        return set_error(FD_ERR_INVALID_ARG, "fd_sparse_create: need nt >= 0 and trace_stride >= npoint");
    // the linear-interpolation cell of a point spans nodes i and i+1 on
    // every axis: an axis of one node has no cell
    for (int a = 0; a < g->ndim && npoint > 0; a++)
        if (g->shape[a] < 2)
            return set_error(FD_ERR_INVALID_ARG, "fd_sparse_create: axis %d has %lld node(s); points need >= 2", a,
                             (long long)g->shape[a]);
    const int ndim = g->ndim;
    std::vector<int64_t> base((size_t)npoint);
    std::vector<float> weight((size_t)npoint * 8, 0.0f);
    fd_status ts = linear_table(*g, npoint, coords, base.data(), weight.data(), "fd_sparse_create");
    if (ts != FD_OK) return ts;
    fd_sparse *sp = new (std::nothrow) fd_sparse();
    if (!sp) return set_error(FD_ERR_NOMEM, "fd_sparse_create: out of host memory");
    sp->g = *g;
    sp->npoint = npoint;
    sp->trace = (float *)dev_trace;
    sp->nt = nt;
    sp->stride = trace_stride;
    sp->alloc_stream = (cudaStream_t)cuda_stream;
    sp->d_base = nullptr;
    sp->d_weight = nullptr;
    if (npoint > 0) {
        cudaStream_t s = sp->alloc_stream;
        cudaError_t e = cudaMallocAsync((void **)&sp->d_base, sizeof(int64_t) * npoint, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&sp->d_weight, sizeof(float) * 8 * npoint, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sp->d_base, base.data(), sizeof(int64_t) * npoint, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sp->d_weight, weight.data(), sizeof(float) * 8 * npoint,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            if (sp->d_base) cudaFreeAsync(sp->d_base, s);
            if (sp->d_weight) cudaFreeAsync(sp->d_weight, s);
            delete sp;
            return e == cudaErrorMemoryAllocation ? set_error(FD_ERR_NOMEM, "fd_sparse_create: device allocation")
                                                  : cuda_error(e, "fd_sparse_create");
        }
    }
    sp->h_base = std::move(base);
    sp->h_weight = std::move(weight);
    SparseDev &d = sp->dev;
    d.npoint = npoint;
    d.ncorner = 1 << ndim;
    d.base = sp->d_base;
    d.weight = sp->d_weight;
    corner_offsets(*g, d.corner_off);
    *out = sp;
    return FD_OK;
}

extern "C" fd_status fd_sparse_set_trace(fd_sparse *sp, void *dev_trace, int64_t nt, int64_t trace_stride)
{
    if (!sp) return set_error(FD_ERR_INVALID_ARG, "fd_sparse_set_trace: null handle");
    if (sp->npoint > 0 && (!dev_trace || trace_stride < sp->npoint || nt < 0))
        return set_error(FD_ERR_INVALID_ARG, "fd_sparse_set_trace: bad trace");
    sp->trace = (float *)dev_trace;
    sp->nt = nt;
    sp->stride = trace_stride;
    return FD_OK;
}

extern "C" void fd_sparse_destroy(fd_sparse *sp)
{
    if (!sp) return;
    if (sp->d_base) cudaFreeAsync(sp->d_base, sp->alloc_stream);
    if (sp->d_weight) cudaFreeAsync(sp->d_weight, sp->alloc_stream);
    delete sp;
}

// ---------------------------------------------------------------------------
// operator
// ---------------------------------------------------------------------------

static fd_status build_coef(fd_operator *op)
{
    double w[9];
    fd_status s = fd_weights_central2(op->so, w);
    if (s != FD_OK) return s;
    const int M = op->so / 2;
    const fd_grid &g = op->u->g;
    Coef &cf = op->coef;
    std::memset(&cf, 0, sizeof cf);
    double centre = 0.0, lam = 0.0;
    double smax = symbol_max(w, M);
    for (int d = 0; d < g.ndim; d++) {
        int a = 3 - g.ndim + d;
        double h2 = g.spacing[d] * g.spacing[d];
        for (int k = 1; k <= M; k++) cf.ax[a][k] = (float)(w[k] / h2);
        cf.ax[a][0] = (float)(w[0] / h2);
        centre += w[0] / h2;
        lam += smax / h2;
    }
    cf.centre = (float)centre;
    op->lambda_max = lam;
    return FD_OK;
}

static fd_status reduce_m_min(fd_operator *op)
{
    unsigned int *d_bits = nullptr;
    unsigned int init = 0x7f7fffffu;  // FLT_MAX
    unsigned int bits = 0;
    FD_CUDA(cudaMallocAsync((void **)&d_bits, sizeof(unsigned int), op->stream), "min(m): cudaMallocAsync");
    cudaError_t e = cudaMemcpyAsync(d_bits, &init, sizeof init, cudaMemcpyHostToDevice, op->stream);
    if (e == cudaSuccess) e = launch_min_reduce(op->geom, op->m->slot[0], d_bits, op->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, d_bits, sizeof bits, cudaMemcpyDeviceToHost, op->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->stream);
    cudaFreeAsync(d_bits, op->stream);
    if (e != cudaSuccess) return cuda_error(e, "min(m)");
    op->launches += 1;
    float mmin;
    std::memcpy(&mmin, &bits, sizeof mmin);
    op->m_min = (double)mmin;
    if (!(op->m_min > 0.0)) return set_error(FD_ERR_INVALID_ARG, "fd_operator: m must be positive everywhere");
    return FD_OK;
}

static fd_status rebuild_fused(fd_operator *op)
{
    if (!op->tma.ready && !op->pair.ready) return FD_OK;
    SparseHostView sv;
    const SparseHostView *sp = nullptr;
    if (op->src && op->src->npoint > 0) {
        sv.npoint = op->src->npoint;
        sv.base = op->src->h_base.data();
        sv.weight = op->src->h_weight.data();
        sp = &sv;
    }
    fd_status s = op->tma.ready ? tma_sparse_build(op->tma, sp, op->stream) : FD_OK;
    if (s == FD_OK && op->pair.ready) s = pair_sparse_build(op->pair, sp, op->stream);
    return s;
}

// Steps per sweep of the acoustic operator: 2 when the two-step kernel is
// planned, fuses every source and is wanted (forced, or the planner's
// default), else 1.
static int acoustic_steps_per_sweep(const fd_operator *op)
{
    if (op->kind != FD_ACOUSTIC_LEAPFROG || !op->pair.ready || !op->tma.ready ||
        (op->flags & FD_FLAG_PLAIN_KERNELS))
        return 1;
    if (op->src && op->src->npoint > 0 && !op->pair.has_src) return 1;
    return op->want_sweep == 2 ? 2 : 1;
}

static void profile_clear(fd_operator *op)
{
    for (cudaEvent_t e : op->prof_ev) cudaEventDestroy(e);
    op->prof_ev.clear();
    op->prof_max = 0;
    op->prof_used = 0;
}

// Record the start (which = 0) or stop (which = 1) event of a profiled launch.
static cudaError_t profile_mark(fd_operator *op, int which)
{
    if (op->prof_used >= op->prof_max) return cudaSuccess;
    cudaEvent_t e = op->prof_ev[(size_t)(2 * op->prof_used + which)];
    cudaError_t r = cudaEventRecord(e, op->stream);
    if (which == 1) op->prof_used += 1;
    return r;
}

// The whole-run cluster plan of a 2D diffusion, convection or Laplace
// operator (none for other kinds or grids that do not fit).
static void plan_cluster(fd_operator *op)
{
    op->cluster = ClusterPlan();
    int rule = -1, M = 1;
    if (op->kind == FD_DIFFUSION_EULER) {
        rule = kRuleDiffusion;
        M = op->so / 2;
    } else if (op->kind == FD_CONVECTION_UPWIND) {
        rule = kRuleUpwind;
    } else if (op->kind == FD_LAPLACE_JACOBI) {
        rule = kRuleJacobi;
    }
    if (rule >= 0) cluster_plan_build(rule, M, op->geom, op->want_k, &op->cluster);
}

static void release(fd_operator *op)
{
    if (!op) return;
    if (op->conv_res) cudaFreeAsync(op->conv_res, op->stream);
    profile_clear(op);
    if (op->side) {
        cudaStreamSynchronize(op->side);
        cudaStreamDestroy(op->side);
    }
    if (op->ev_u) cudaEventDestroy(op->ev_u);
    if (op->ev_rec) cudaEventDestroy(op->ev_rec);
    if (op->c) cudaFreeAsync(op->c, op->stream);
    if (op->d) cudaFreeAsync(op->d, op->stream);
    if (op->status) cudaFreeAsync(op->status, op->stream);
    tma_plan_release(op->tma, op->stream);
    pair_plan_release(op->pair, op->stream);
    delete op;
}

extern "C" fd_status fd_operator_create(const fd_op_desc *desc, fd_operator **out)
{
    if (!desc || !out) return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: null pointer");
    *out = nullptr;
    const int kind = desc->kind;
    if (kind != FD_DIFFUSION_EULER && kind != FD_ACOUSTIC_LEAPFROG && kind != FD_CONVECTION_UPWIND &&
        kind != FD_LAPLACE_JACOBI)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: unknown kind %d", kind);
    if (kind == FD_CONVECTION_UPWIND && desc->space_order != 1)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: convection is first order (space_order 1)");
    if (kind == FD_LAPLACE_JACOBI && desc->space_order != 2)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: the Laplace sweep is second order (space_order 2)");
    if (kind != FD_CONVECTION_UPWIND &&
        (desc->space_order < 2 || desc->space_order > 16 || desc->space_order % 2))
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: space order must be even, 2..16");
    if (!desc->u || desc->u->levels != 2)
        return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: u must be a 2-slot field");
    const fd_grid &g = desc->u->g;
    if ((kind == FD_CONVECTION_UPWIND || kind == FD_LAPLACE_JACOBI) && g.ndim != 2)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: the convection and Laplace operators are 2D");
    if (kind == FD_LAPLACE_JACOBI && (g.shape[0] < 3 || g.shape[1] < 3))
        return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: the Laplace sweep needs at least 3 x 3 nodes");
    if (desc->kind == FD_ACOUSTIC_LEAPFROG) {
        if (!desc->m || desc->m->levels != 1 || !same_shape(desc->m->g, g))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: acoustic needs a 1-slot m of u's shape");
        if (desc->eta && (desc->eta->levels != 1 || !same_shape(desc->eta->g, g)))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: eta must be a 1-slot field of u's shape");
        if ((desc->src && !same_shape(desc->src->g, g)) || (desc->rec && !same_shape(desc->rec->g, g)))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: sparse grid differs from u's");
    } else {
        if (kind != FD_LAPLACE_JACOBI && (!(desc->a > 0.0) || !std::isfinite(desc->a)))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_create: %s must be > 0",
                             kind == FD_CONVECTION_UPWIND ? "velocity c (a)" : "diffusivity a");
        if (desc->flags & FD_FLAG_REVERSE)
            return set_error(FD_ERR_UNSUPPORTED, "fd_operator_create: only the acoustic operator has a reverse mode");
    }
    fd_operator *op = new (std::nothrow) fd_operator();
    if (!op) return set_error(FD_ERR_NOMEM, "fd_operator_create: out of host memory");
    op->kind = desc->kind;
    op->so = desc->space_order;
    op->u = desc->u;
    op->m = desc->m;
    op->eta = desc->eta;
    op->a = desc->a;
    op->src = desc->kind == FD_ACOUSTIC_LEAPFROG ? desc->src : nullptr;
    op->rec = desc->kind == FD_ACOUSTIC_LEAPFROG ? desc->rec : nullptr;
    op->stream = (cudaStream_t)desc->cuda_stream;
    op->flags = desc->flags;
    op->geom = geom_of(g);
    op->c = op->d = nullptr;
    op->status = nullptr;
    op->coef_dt = -1.0;
    op->m_min = 0.0;
    op->launches = 0;
    op->prof_max = 0;
    op->prof_used = 0;
    op->want_k = 0;
    op->want_sweep = 0;
    op->side = nullptr;
    op->ev_u = op->ev_rec = nullptr;
    op->jac_wr = op->jac_wc = 0.0f;
    op->conv_res = nullptr;
    std::memset(&op->coef, 0, sizeof op->coef);
    op->lambda_max = 0.0;
    fd_status s = op->kind == FD_CONVECTION_UPWIND ? FD_OK : build_coef(op);
    if (s != FD_OK) { release(op); return s; }
    if (op->kind == FD_LAPLACE_JACOBI) {
        // central second differences solved for the centre: the row (x)
        // neighbours weigh dy^2, the column (y) neighbours dx^2, over 2(dx^2+dy^2)
        const double hx2 = g.spacing[0] * g.spacing[0], hy2 = g.spacing[1] * g.spacing[1];
        op->jac_wr = (float)(hy2 / (2.0 * (hx2 + hy2)));
        op->jac_wc = (float)(hx2 / (2.0 * (hx2 + hy2)));
        cudaError_t e2 = cudaMallocAsync(&op->conv_res, 32, op->stream);
        if (e2 != cudaSuccess) { release(op); return cuda_error(e2, "fd_operator_create: result word"); }
    }
    cudaError_t e = cudaMallocAsync((void **)&op->status, sizeof(int), op->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(op->status, 0, sizeof(int), op->stream);
    if (e != cudaSuccess) { release(op); return cuda_error(e, "fd_operator_create: status word"); }
    if (op->kind == FD_ACOUSTIC_LEAPFROG) {
        size_t bytes = sizeof(float) * (size_t)slot_elems(g);
        e = cudaMallocAsync((void **)&op->c, bytes, op->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&op->d, bytes, op->stream);
        if (e != cudaSuccess) {
            release(op);
            return e == cudaErrorMemoryAllocation ? set_error(FD_ERR_NOMEM, "fd_operator_create: coefficient fields")
                                                  : cuda_error(e, "fd_operator_create");
        }
        s = reduce_m_min(op);
        if (s != FD_OK) { release(op); return s; }
    }
    s = tma_plan_build(op->tma, op->kind, op->so, op->geom, op->u->slot, op->c, op->d);
    if (s != FD_OK) { release(op); return s; }
    if (op->kind == FD_ACOUSTIC_LEAPFROG && op->tma.ready) {
        s = pair_plan_build(op->pair, op->so, op->geom, op->u->slot, op->c, op->d);
        if (s != FD_OK) { release(op); return s; }
    }
    s = rebuild_fused(op);
    if (s != FD_OK) { release(op); return s; }
    plan_cluster(op);
    *out = op;
    return FD_OK;
}

extern "C" fd_status fd_operator_bind(fd_operator *op, const char *name, void *obj)
{
    if (!op || !name) return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: null pointer");
    const fd_grid &g = op->u->g;
    std::string n(name);
    if (n == "u") {
        fd_field *f = (fd_field *)obj;
        if (!f || f->levels != 2 || !same_shape(f->g, g))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: u must be a 2-slot field of the same shape");
        op->u = f;
        // the rebuilt plan stages no injected corners until the fused table
        // is rebuilt for it
        fd_status s = tma_plan_build(op->tma, op->kind, op->so, op->geom, op->u->slot, op->c, op->d);
        if (s == FD_OK && op->pair.ready)
            s = pair_plan_build(op->pair, op->so, op->geom, op->u->slot, op->c, op->d);
        return s != FD_OK ? s : rebuild_fused(op);
    }
    if (n == "m" || n == "eta") {
        if (op->kind != FD_ACOUSTIC_LEAPFROG)
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: %s only for the acoustic operator", name);
        fd_field *f = (fd_field *)obj;
        if ((n == "m" && !f) || (f && (f->levels != 1 || !same_shape(f->g, g))))
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: %s must be a 1-slot field of u's shape", name);
        if (n == "m") {
            op->m = f;
            fd_status s = reduce_m_min(op);
            if (s != FD_OK) return s;
        } else {
            op->eta = f;
        }
        op->coef_dt = -1.0;
        return FD_OK;
    }
    if (n == "src" || n == "rec") {
        fd_sparse *sp = (fd_sparse *)obj;
        if (sp && !same_shape(sp->g, g)) return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: sparse grid differs");
        if (op->kind != FD_ACOUSTIC_LEAPFROG && sp)
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: sparse points only for the acoustic operator");
        (n == "src" ? op->src : op->rec) = sp;
        return rebuild_fused(op);
    }
    if (n == "stream") {
        op->stream = (cudaStream_t)obj;
        return FD_OK;
    }
    if (n == "a") {
        const double *a = (const double *)obj;
        if (!a || !(*a > 0.0)) return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: a must be > 0");
        op->a = *a;
        return FD_OK;
    }
    return set_error(FD_ERR_INVALID_ARG, "fd_operator_bind: unknown name '%s'", name);
}

// Stability check of fd_operator_apply / fd_operator_step.
static fd_status check_dt(const fd_operator *op, double dt, const char *who)
{
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_error(FD_ERR_INVALID_ARG, "%s: dt must be > 0", who);
    if (op->flags & FD_FLAG_NO_CFL_CHECK) return FD_OK;
    if (op->kind == FD_CONVECTION_UPWIND) {
        const fd_grid &g = op->u->g;
        const double nu = op->a * dt * (1.0 / g.spacing[0] + 1.0 / g.spacing[1]);
        if (nu > 1.0)
            return set_error(FD_ERR_UNSTABLE, "%s: c dt (1/dx + 1/dy) = %g above the upwind limit 1", who, nu);
        return FD_OK;
    }
    if (op->kind == FD_ACOUSTIC_LEAPFROG) {
        double limit = 2.0 * std::sqrt(op->m_min / op->lambda_max);
        if (dt > limit) return set_error(FD_ERR_UNSTABLE, "%s: dt = %g above the stability limit %g", who, dt, limit);
    } else {
        double limit = 2.0 / (op->a * op->lambda_max);
        if (dt > limit)
            return set_error(FD_ERR_UNSTABLE, "%s: a*dt = %g above the Euler limit %g", who, op->a * dt, op->a * limit);
    }
    return FD_OK;
}

// Recompute c, d (and the damping flags of the tiled kernel) when dt or the
// inputs changed.
static fd_status prepare_coefficients(fd_operator *op, double dt)
{
    if (op->kind != FD_ACOUSTIC_LEAPFROG || op->coef_dt == dt) return FD_OK;
    cudaStream_t st = op->stream;
    FD_CUDA(launch_coefficients(op->geom, op->m->slot[0], op->eta ? op->eta->slot[0] : nullptr, dt, op->c, op->d, st),
            "coefficients");
    op->launches += 1;
    op->coef_dt = dt;
    return FD_OK;
}

// Receivers of step n read u^n while the update of step n writes the other
// slot, so the interpolation runs on a side stream beside the update; the
// operator's stream waits for it before the next update (which overwrites
// u^n) and at the end of the call.
static cudaError_t interpolate_beside(fd_operator *op, const float *u, float *rec_row)
{
    cudaError_t e = cudaSuccess;
    if (!op->side) {
        e = cudaStreamCreateWithFlags(&op->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&op->ev_u, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&op->ev_rec, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(op->ev_u, op->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(op->side, op->ev_u, 0);
    if (e == cudaSuccess) e = launch_interpolate(op->rec->dev, u, rec_row, op->side);
    if (e == cudaSuccess) e = cudaEventRecord(op->ev_rec, op->side);
    return e;
}

// The time loop of fd_operator_apply; with `img`, every step also
// accumulates the imaging condition from the field it writes -- fused into
// the tiled kernel when that kernel fuses the step's sources too, else as a
// separate kernel after the step (and its injection).
static fd_status apply_steps(fd_operator *op, int64_t t0, int64_t nt, double dt, const ImagingArgs *img)
{
    if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply: null operator");
    if (nt < 0 || t0 < 0) return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply: need t0 >= 0, nt >= 0");
    const bool reverse = (op->flags & FD_FLAG_REVERSE) != 0;
    for (fd_sparse *sp : {op->src, op->rec})
        if (sp && sp->npoint > 0 && t0 + nt > sp->nt)
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply: trace has %lld rows, need %lld",
                             (long long)sp->nt, (long long)(t0 + nt));
    fd_status cs = op->kind == FD_LAPLACE_JACOBI ? FD_OK : check_dt(op, dt, "fd_operator_apply");
    if (cs != FD_OK) return cs;
    if (nt == 0) return FD_OK;
    const int M = op->so / 2;
    const Geom &g = op->geom;
    cudaStream_t st = op->stream;
    const bool plain = (op->flags & FD_FLAG_PLAIN_KERNELS) != 0 || !op->tma.ready;
    if (op->kind == FD_ACOUSTIC_LEAPFROG) {
        cs = prepare_coefficients(op, dt);
        if (cs != FD_OK) return cs;
        const int sweep = plain ? 1 : acoustic_steps_per_sweep(op);
        const bool has_rec = op->rec && op->rec->npoint > 0, has_src = op->src && op->src->npoint > 0;
        // receivers beside the update only for runs of many steps: a call of
        // one step has nothing to overlap and would pay the two cross-stream
        // dependencies per step (a step-by-step adjoint, for instance)
        const bool beside = nt >= 16;
        for (int64_t q = 0; q < nt; q++) {
            int64_t n = reverse ? t0 + nt - 1 - q : t0 + q;
            int cur = (int)((reverse ? n + 1 : n) & 1);
            float *u = op->u->slot[cur];
            float *up = op->u->slot[cur ^ 1];
            float *rec_row = has_rec ? op->rec->trace + n * op->rec->stride : nullptr;
            const float *src_row = has_src ? op->src->trace + n * op->src->stride : nullptr;
            if (sweep == 2 && nt - q >= 2) {
                // steps n and n2 in one sweep: receivers of n read u^n before
                // it, those of n2 read u^{n+1} (the buffer of u^{n-1}) after it
                const int64_t n2 = reverse ? n - 1 : n + 1;
                if (rec_row) {
                    FD_CUDA(launch_interpolate(op->rec->dev, u, rec_row, st), "interpolate");
                    op->launches += 1;
                }
                FD_CUDA(profile_mark(op, 0), "profile");
                FD_CUDA(launch_acoustic_pair(op->pair, op->coef, cur, op->status, src_row,
                                             has_src ? op->src->trace + n2 * op->src->stride : nullptr, st),
                        "two-step sweep");
                FD_CUDA(profile_mark(op, 1), "profile");
                op->launches += 1;
                if (has_rec) {
                    FD_CUDA(launch_interpolate(op->rec->dev, up, op->rec->trace + n2 * op->rec->stride, st),
                            "interpolate");
                    op->launches += 1;
                }
                q++;
                continue;
            }
            if (plain) {
                if (rec_row) {
                    FD_CUDA(launch_interpolate(op->rec->dev, u, rec_row, st), "interpolate");
                    op->launches += 1;
                }
                FD_CUDA(profile_mark(op, 0), "profile");
                FD_CUDA(launch_acoustic_plain(M, g, op->coef, u, up, up, op->c, op->d, st), "acoustic step");
                FD_CUDA(profile_mark(op, 1), "profile");
                op->launches += 1;
                if (src_row) {
                    FD_CUDA(launch_inject(op->src->dev, op->c, src_row, up, st), "inject");
                    op->launches += 1;
                }
                if (img) {
                    FD_CUDA(launch_imaging(g, img->scale, up, img->u0, img->u1, img->u2, img->grad, st), "imaging");
                    op->launches += 1;
                }
            } else {
                // receivers: a small kernel reading u^n, beside the update;
                // sources: fused into the tiled kernel when the per-tile
                // lists fit in shared memory
                if (rec_row) {
                    if (beside)
                        FD_CUDA(interpolate_beside(op, u, rec_row), "interpolate");
                    else
                        FD_CUDA(launch_interpolate(op->rec->dev, u, rec_row, st), "interpolate");
                    op->launches += 1;
                }
                // the imaging condition rides in the sweep when the value the
                // sweep writes is final (sources fused or absent)
                const bool fuse_img = img && (!src_row || op->tma.has_src);
                FD_CUDA(profile_mark(op, 0), "profile");
                if (fuse_img)
                    FD_CUDA(launch_acoustic_tma_imaging(op->tma, M, op->coef, cur, op->status, src_row, *img, st),
                            "acoustic step with imaging");
                else
                    FD_CUDA(launch_acoustic_tma(op->tma, M, g, op->coef, cur, op->status, src_row, st),
                            "acoustic step");
                FD_CUDA(profile_mark(op, 1), "profile");
                op->launches += 1;
                if (rec_row && beside) FD_CUDA(cudaStreamWaitEvent(st, op->ev_rec, 0), "interpolate");
                if (src_row && !op->tma.has_src) {
                    FD_CUDA(launch_inject(op->src->dev, op->c, src_row, up, st), "inject");
                    op->launches += 1;
                }
                if (img && !fuse_img) {
                    FD_CUDA(launch_imaging(g, img->scale, up, img->u0, img->u1, img->u2, img->grad, st), "imaging");
                    op->launches += 1;
                }
            }
        }
    } else {
        // 2D diffusion, convection and Laplace sweeps: the whole run in one
        // cluster launch when the grid fits, else one launch per step
        const fd_grid &gr = op->u->g;
        const float adt = (float)(op->a * dt);
        const float nux = op->kind == FD_CONVECTION_UPWIND ? (float)(op->a * dt / gr.spacing[0]) : 0.0f;
        const float nuy = op->kind == FD_CONVECTION_UPWIND ? (float)(op->a * dt / gr.spacing[1]) : 0.0f;
        if (op->cluster.ok && !(op->flags & FD_FLAG_PLAIN_KERNELS)) {
            FD_CUDA(profile_mark(op, 0), "profile");
            FD_CUDA(launch_cluster_run(op->cluster, g, op->coef, adt, nux, nuy, op->jac_wr, op->jac_wc,
                                       op->u->slot[t0 & 1], op->u->slot[0], op->u->slot[1], t0, nt, 0.0, nullptr,
                                       nullptr, st),
                    "cluster run");
            FD_CUDA(profile_mark(op, 1), "profile");
            op->launches += 1;
        } else {
            for (int64_t q = 0; q < nt; q++) {
                int64_t n = t0 + q;
                int cur = (int)(n & 1);
                const float *src = op->u->slot[cur];
                float *dst = op->u->slot[cur ^ 1];
                FD_CUDA(profile_mark(op, 0), "profile");
                if (op->kind == FD_DIFFUSION_EULER)
                    FD_CUDA(launch_diffusion_plain(M, g, op->coef, adt, src, dst, st), "diffusion step");
                else if (op->kind == FD_CONVECTION_UPWIND)
                    FD_CUDA(launch_convection_plain(g, nux, nuy, src, dst, st), "convection step");
                else
                    FD_CUDA(launch_jacobi_plain(g, op->jac_wr, op->jac_wc, src, dst, nullptr, st), "Laplace sweep");
                FD_CUDA(profile_mark(op, 1), "profile");
                op->launches += 1;
            }
        }
    }
    return FD_OK;
}

extern "C" fd_status fd_operator_apply(fd_operator *op, int64_t t0, int64_t nt, double dt)
{
    return apply_steps(op, t0, nt, dt, nullptr);
}

extern "C" fd_status fd_operator_apply_imaging(fd_operator *op, int64_t n, double dt, double scale, const void *u0,
                                               const void *u1, const void *u2, void *grad)
{
    if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply_imaging: null operator");
    if (op->kind != FD_ACOUSTIC_LEAPFROG)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_apply_imaging: acoustic operators only");
    if (!u0 || !u1 || !u2 || !grad) return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply_imaging: null buffer");
    for (const void *p : {u0, u1, u2, (const void *)grad})
        if (((uintptr_t)p) % 32 != 0)
            return set_error(FD_ERR_LAYOUT, "fd_operator_apply_imaging: buffer not 32-byte aligned");
    for (const void *p : {u0, u1, u2, (const void *)grad})
        if (p == op->u->slot[0] || p == op->u->slot[1])
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply_imaging: a buffer is a slot of the operator's field");
    if (!std::isfinite(scale)) return set_error(FD_ERR_INVALID_ARG, "fd_operator_apply_imaging: scale not finite");
    ImagingArgs img;
    img.u0 = (const float *)u0;
    img.u1 = (const float *)u1;
    img.u2 = (const float *)u2;
    img.grad = (float *)grad;
    img.scale = (float)scale;
    return apply_steps(op, n, 1, dt, &img);
}

extern "C" fd_status fd_operator_sync(fd_operator *op)
{
    if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_operator_sync: null operator");
    FD_CUDA(cudaStreamSynchronize(op->stream), "fd_operator_sync");
    FD_CUDA(cudaGetLastError(), "fd_operator_sync");
    int status = 0;
    FD_CUDA(cudaMemcpy(&status, op->status, sizeof status, cudaMemcpyDeviceToHost), "fd_operator_sync: status");
    if (status != 0) {
        cudaMemset(op->status, 0, sizeof(int));
        cudaDeviceSynchronize();
        return set_error(FD_ERR_TIMEOUT, "fd_operator_sync: a device wait gave up (code %d)", status);
    }
    return FD_OK;
}

extern "C" void fd_operator_destroy(fd_operator *op) { release(op); }

extern "C" int64_t fd_operator_launch_count(const fd_operator *op) { return op ? op->launches : 0; }

extern "C" fd_status fd_operator_profile(fd_operator *op, int64_t max_launches)
{
    if (!op || max_launches < 0 || max_launches > (int64_t(1) << 20))
        return set_error(FD_ERR_INVALID_ARG, "fd_operator_profile: bad arguments");
    FD_CUDA(cudaStreamSynchronize(op->stream), "fd_operator_profile");
    profile_clear(op);
    try {
        op->prof_ev.resize((size_t)(2 * max_launches), nullptr);
    } catch (...) {
        return set_error(FD_ERR_NOMEM, "fd_operator_profile: out of host memory");
    }
    for (auto &e : op->prof_ev) {
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) {
            e = nullptr;
            profile_clear(op);
            return cuda_error(r, "fd_operator_profile: cudaEventCreate");
        }
    }
    op->prof_max = max_launches;
    op->prof_used = 0;
    return FD_OK;
}

extern "C" fd_status fd_operator_profile_read(fd_operator *op, double *total_ms, int64_t *launches)
{
    if (!op || !total_ms || !launches) return set_error(FD_ERR_INVALID_ARG, "fd_operator_profile_read: null pointer");
    FD_CUDA(cudaStreamSynchronize(op->stream), "fd_operator_profile_read");
    double sum = 0.0;
    for (int64_t i = 0; i < op->prof_used; i++) {
        float ms = 0.0f;
        FD_CUDA(cudaEventElapsedTime(&ms, op->prof_ev[(size_t)(2 * i)], op->prof_ev[(size_t)(2 * i + 1)]),
                "fd_operator_profile_read");
        sum += ms;
    }
    *total_ms = sum;
    *launches = op->prof_used;
    return FD_OK;
}

extern "C" fd_status fd_operator_step(fd_operator *op, int64_t n, double dt, const void *u_cur, const void *u_prev,
                                      void *u_next)
{
    if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_operator_step: null operator");
    if (op->kind != FD_ACOUSTIC_LEAPFROG)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_step: acoustic operators only");
    if (!u_cur || !u_prev || !u_next) return set_error(FD_ERR_INVALID_ARG, "fd_operator_step: null buffer");
    if (u_next == u_cur) return set_error(FD_ERR_INVALID_ARG, "fd_operator_step: u_next must differ from u_cur");
    for (const void *p : {u_cur, u_prev, (const void *)u_next})
        if (((uintptr_t)p) % 32 != 0) return set_error(FD_ERR_LAYOUT, "fd_operator_step: buffer not 32-byte aligned");
    if (n < 0) return set_error(FD_ERR_INVALID_ARG, "fd_operator_step: n < 0");
    for (fd_sparse *sp : {op->src, op->rec})
        if (sp && sp->npoint > 0 && n >= sp->nt)
            return set_error(FD_ERR_INVALID_ARG, "fd_operator_step: trace has %lld rows, need row %lld",
                             (long long)sp->nt, (long long)n);
    fd_status cs = check_dt(op, dt, "fd_operator_step");
    if (cs != FD_OK) return cs;
    cs = prepare_coefficients(op, dt);
    if (cs != FD_OK) return cs;
    const int M = op->so / 2;
    cudaStream_t st = op->stream;
    const float *uc = (const float *)u_cur;
    const float *up = (const float *)u_prev;
    float *un = (float *)u_next;
    float *rec_row = (op->rec && op->rec->npoint > 0) ? op->rec->trace + n * op->rec->stride : nullptr;
    const float *src_row = (op->src && op->src->npoint > 0) ? op->src->trace + n * op->src->stride : nullptr;
    const bool plain = (op->flags & FD_FLAG_PLAIN_KERNELS) != 0 || !op->tma.ready;
    if (plain) {
        if (rec_row) {
            FD_CUDA(launch_interpolate(op->rec->dev, uc, rec_row, st), "interpolate");
            op->launches += 1;
        }
        FD_CUDA(profile_mark(op, 0), "profile");
        FD_CUDA(launch_acoustic_plain(M, op->geom, op->coef, uc, up, un, op->c, op->d, st), "acoustic step");
        FD_CUDA(profile_mark(op, 1), "profile");
        op->launches += 1;
        if (src_row) {
            FD_CUDA(launch_inject(op->src->dev, op->c, src_row, un, st), "inject");
            op->launches += 1;
        }
    } else {
        if (rec_row) {
            FD_CUDA(launch_interpolate(op->rec->dev, uc, rec_row, st), "interpolate");
            op->launches += 1;
        }
        FD_CUDA(profile_mark(op, 0), "profile");
        FD_CUDA(launch_acoustic_tma_buffers(op->tma, M, op->coef, uc, up, un, op->status, src_row, st),
                "acoustic step");
        FD_CUDA(profile_mark(op, 1), "profile");
        op->launches += 1;
        if (src_row && !op->tma.has_src) {
            FD_CUDA(launch_inject(op->src->dev, op->c, src_row, un, st), "inject");
            op->launches += 1;
        }
    }
    return FD_OK;
}

extern "C" fd_status fd_imaging_accumulate(const fd_grid *g, double scale, const void *mu, const void *u0,
                                           const void *u1, const void *u2, void *grad, void *cuda_stream)
{
    if (!g || !mu || !u0 || !u1 || !u2 || !grad)
        return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate: null pointer");
    for (const void *p : {mu, u0, u1, u2, (const void *)grad})
        if (((uintptr_t)p) % 16 != 0) return set_error(FD_ERR_LAYOUT, "fd_imaging_accumulate: buffer not aligned");
    FD_CUDA(launch_imaging(geom_of(*g), (float)scale, (const float *)mu, (const float *)u0, (const float *)u1,
                           (const float *)u2, (float *)grad, (cudaStream_t)cuda_stream),
            "fd_imaging_accumulate");
    return FD_OK;
}

extern "C" fd_status fd_imaging_accumulate_steps(const fd_grid *g, double scale, int k, const void *const *mu,
                                                 const void *const *u, void *grad, void *cuda_stream)
{
    if (!g || !mu || !u || !grad) return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate_steps: null pointer");
    if (k < 1 || k > 4) return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate_steps: k = %d (1..4)", k);
    const float *pm[4] = {};
    const float *pu[6] = {};
    for (int i = 0; i < k + 2; i++) {
        const void *q[2] = {i < k ? mu[i] : nullptr, u[i]};
        for (int s = 0; s < 2; s++) {
            if (s == 0 && i >= k) continue;
            if (!q[s]) return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate_steps: null buffer");
            if (((uintptr_t)q[s]) % 16 != 0)
                return set_error(FD_ERR_LAYOUT, "fd_imaging_accumulate_steps: buffer not aligned");
            if (q[s] == grad) return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate_steps: grad aliases an input");
        }
        if (i < k) pm[i] = (const float *)mu[i];
        pu[i] = (const float *)u[i];
    }
    if (((uintptr_t)grad) % 16 != 0) return set_error(FD_ERR_LAYOUT, "fd_imaging_accumulate_steps: grad not aligned");
    if (!std::isfinite(scale)) return set_error(FD_ERR_INVALID_ARG, "fd_imaging_accumulate_steps: scale not finite");
    FD_CUDA(launch_imaging_steps(geom_of(*g), (float)scale, k, pm, pu, (float *)grad, (cudaStream_t)cuda_stream),
            "fd_imaging_accumulate_steps");
    return FD_OK;
}

extern "C" fd_status fd_operator_debug_stall(fd_operator *op, int plane)
{
    if (!op || plane < -1) return set_error(FD_ERR_INVALID_ARG, "fd_operator_debug_stall: bad arguments");
    if (!op->tma.ready) return set_error(FD_ERR_UNSUPPORTED, "fd_operator_debug_stall: no tiled kernel");
    op->tma.stall_plane = plane;
    op->tma.args.stall_plane = plane;
    op->pair.args.stall_plane = plane;
    return FD_OK;
}

extern "C" fd_status fd_operator_set_tiling(fd_operator *op, int rows, int stages)
{
    if (!op || rows < 0 || stages < 0) return set_error(FD_ERR_INVALID_ARG, "fd_operator_set_tiling: bad arguments");
    if (!op->tma.ready && (rows > 0 || stages > 0))
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_set_tiling: this operator has no tiled kernel");
    FD_CUDA(cudaStreamSynchronize(op->stream), "fd_operator_set_tiling");
    const int old_rows = op->tma.force_rows, old_stages = op->tma.force_stages;
    op->tma.force_rows = rows;
    op->tma.force_stages = stages;
    op->tma.cache.clear();
    fd_status s = tma_plan_build(op->tma, op->kind, op->so, op->geom, op->u->slot, op->c, op->d);
    if (s != FD_OK) {
        op->tma.force_rows = old_rows;
        op->tma.force_stages = old_stages;
        tma_plan_build(op->tma, op->kind, op->so, op->geom, op->u->slot, op->c, op->d);
        rebuild_fused(op);
        return s;
    }
    return rebuild_fused(op);
}

extern "C" fd_status fd_operator_get_tiling(const fd_operator *op, int *rows, int *stages, int *ctas)
{
    if (!op || !rows || !stages || !ctas) return set_error(FD_ERR_INVALID_ARG, "fd_operator_get_tiling: null pointer");
    tma_plan_tiling(op->tma, rows, stages, ctas);
    return FD_OK;
}

extern "C" fd_status fd_operator_sources_fused(const fd_operator *op, int *fused)
{
    if (!op || !fused) return set_error(FD_ERR_INVALID_ARG, "fd_operator_sources_fused: null pointer");
    const bool plain = (op->flags & FD_FLAG_PLAIN_KERNELS) != 0 || !op->tma.ready;
    *fused = (!plain && op->tma.has_src && op->src && op->src->npoint > 0) ? 1 : 0;
    return FD_OK;
}

extern "C" fd_status fd_operator_autotune(fd_operator *op, int64_t t0, int64_t nsteps, double dt, int *best_rows,
                                          int *best_stages, double *best_ms_per_step)
{
    if (!op || nsteps < 1 || t0 < 0) return set_error(FD_ERR_INVALID_ARG, "fd_operator_autotune: bad arguments");
    if (!op->tma.ready) return set_error(FD_ERR_UNSUPPORTED, "fd_operator_autotune: no tiled kernel to tune");
    static const int kRows[] = {8, 10, 12, 14, 16, 18, 20, 24, 27, 30};
    cudaEvent_t e0, e1;
    FD_CUDA(cudaEventCreate(&e0), "fd_operator_autotune");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(FD_ERR_CUDA, "fd_operator_autotune: cudaEventCreate");
    }
    int br = 0, bs = 0;
    double bms = 1e30;
    fd_status last = FD_OK;
    for (int rows : kRows) {
        for (int stages = 2; stages <= 4; stages++) {
            // several heights can round to the same balanced strips: time once
            bool seen = false;
            for (int prev : kRows) {
                if (prev >= rows) break;
                if ((op->geom.n[1] + prev - 1) / prev == (op->geom.n[1] + rows - 1) / rows) seen = true;
            }
            if (seen) continue;
            if (fd_operator_set_tiling(op, rows, stages) != FD_OK) continue;
            last = fd_operator_apply(op, t0, nsteps < 3 ? nsteps : 3, dt);  // warm-up, coefficients
            if (last != FD_OK) break;
            cudaEventRecord(e0, op->stream);
            last = fd_operator_apply(op, t0, nsteps, dt);
            cudaEventRecord(e1, op->stream);
            if (last != FD_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                last = set_error(FD_ERR_CUDA, "fd_operator_autotune: timing");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / (double)nsteps;
            if (per < bms) {
                bms = per;
                br = rows;
                bs = stages;
            }
        }
        if (last != FD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (last != FD_OK) return last;
    if (br == 0) return set_error(FD_ERR_UNSUPPORTED, "fd_operator_autotune: no tiling fits");
    fd_status s = fd_operator_set_tiling(op, br, bs);
    if (s != FD_OK) return s;
    if (best_rows) *best_rows = br;
    if (best_stages) *best_stages = bs;
    if (best_ms_per_step) *best_ms_per_step = bms;
    return FD_OK;
}

extern "C" fd_status fd_operator_converge(fd_operator *op, int64_t t0, int64_t max_iter, double tol,
                                          int64_t *iters, double *r_last)
{
    if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_operator_converge: null operator");
    if (op->kind != FD_LAPLACE_JACOBI)
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_converge: only for the Laplace operator");
    if (!(tol > 0.0) || max_iter < 0 || t0 < 0)
        return set_error(FD_ERR_INVALID_ARG, "fd_operator_converge: need tol > 0, max_iter >= 0, t0 >= 0");
    cudaStream_t st = op->stream;
    const Geom &g = op->geom;
    long long steps = 0;
    double r = INFINITY;
    if (max_iter > 0 && op->cluster.ok && !(op->flags & FD_FLAG_PLAIN_KERNELS)) {
        long long *d_steps = (long long *)op->conv_res;
        double *d_r = (double *)((char *)op->conv_res + 8);
        FD_CUDA(launch_cluster_run(op->cluster, g, op->coef, 0.0f, 0.0f, 0.0f, op->jac_wr, op->jac_wc,
                                   op->u->slot[t0 & 1], op->u->slot[0], op->u->slot[1], t0, max_iter, tol, d_steps,
                                   d_r, st),
                "cluster convergence run");
        op->launches += 1;
        unsigned char host[16];
        FD_CUDA(cudaMemcpyAsync(host, op->conv_res, 16, cudaMemcpyDeviceToHost, st), "convergence result");
        FD_CUDA(cudaStreamSynchronize(st), "convergence result");
        std::memcpy(&steps, host, 8);
        std::memcpy(&r, host + 8, 8);
    } else if (max_iter > 0) {
        // per-sweep launches; S read back after every sweep
        double *d_sum = (double *)((char *)op->conv_res + 16);
        double s_old = 0.0, s_new = 0.0;
        FD_CUDA(cudaMemsetAsync(d_sum, 0, sizeof(double), st), "convergence sum");
        FD_CUDA(launch_abs_sum(g, op->u->slot[t0 & 1], d_sum, st), "convergence sum");
        FD_CUDA(cudaMemcpyAsync(&s_old, d_sum, sizeof(double), cudaMemcpyDeviceToHost, st), "convergence sum");
        FD_CUDA(cudaStreamSynchronize(st), "convergence sum");
        op->launches += 1;
        while (steps < max_iter) {
            const int64_t n = t0 + steps;
            FD_CUDA(cudaMemsetAsync(d_sum, 0, sizeof(double), st), "convergence sum");
            FD_CUDA(launch_jacobi_plain(g, op->jac_wr, op->jac_wc, op->u->slot[n & 1], op->u->slot[(n + 1) & 1],
                                        d_sum, st),
                    "Laplace sweep");
            FD_CUDA(cudaMemcpyAsync(&s_new, d_sum, sizeof(double), cudaMemcpyDeviceToHost, st), "convergence sum");
            FD_CUDA(cudaStreamSynchronize(st), "convergence sum");
            op->launches += 1;
            steps++;
            r = s_old > 0.0 ? std::fabs(s_new - s_old) / s_old : INFINITY;
            s_old = s_new;
            if (r < tol) break;
        }
    }
    if (iters) *iters = steps;
    if (r_last) *r_last = r;
    return FD_OK;
}

extern "C" fd_status fd_operator_set_time_block(fd_operator *op, int k)
{
    if (!op || k < 0) return set_error(FD_ERR_INVALID_ARG, "fd_operator_set_time_block: bad arguments");
    if (op->kind == FD_ACOUSTIC_LEAPFROG) {
        if (k > 2) return set_error(FD_ERR_UNSUPPORTED, "fd_operator_set_time_block: 1 or 2 steps per sweep");
        if (k == 2 && (!op->pair.ready || !op->tma.ready || (op->flags & FD_FLAG_PLAIN_KERNELS) ||
                       (op->src && op->src->npoint > 0 && !op->pair.has_src)))
            return set_error(FD_ERR_UNSUPPORTED,
                             "fd_operator_set_time_block: no two-step kernel for this operator (SO 4..8, 3D, "
                             "every column resident, sources fused)");
        op->want_sweep = k;
        return FD_OK;
    }
    if (!op->cluster.ok) return set_error(FD_ERR_UNSUPPORTED, "fd_operator_set_time_block: no cluster path");
    const int old = op->want_k;
    const ClusterPlan keep = op->cluster;
    op->want_k = k;
    plan_cluster(op);
    if (!op->cluster.ok || (k > 0 && op->cluster.nctas > 1 && op->cluster.K != k)) {
        op->want_k = old;
        op->cluster = keep;
        return set_error(FD_ERR_UNSUPPORTED, "fd_operator_set_time_block: %d steps per exchange do not fit", k);
    }
    return FD_OK;
}

extern "C" fd_status fd_operator_get_time_block(const fd_operator *op, int *k, int *ctas)
{
    if (!op || !k || !ctas) return set_error(FD_ERR_INVALID_ARG, "fd_operator_get_time_block: null pointer");
    if (op->kind == FD_ACOUSTIC_LEAPFROG) {
        *k = acoustic_steps_per_sweep(op);
        int rows = 0, stages = 0, c1 = 0;
        tma_plan_tiling(op->tma, &rows, &stages, &c1);
        *ctas = *k == 2 ? op->pair.args.k1 * op->pair.args.k2 : (op->tma.ready ? c1 : 0);
        return FD_OK;
    }
    *k = op->cluster.ok ? op->cluster.K : 0;
    *ctas = op->cluster.ok ? op->cluster.nctas : 0;
    return FD_OK;
}

// ---------------------------------------------------------------------------
// batches of shots
// ---------------------------------------------------------------------------

struct fd_batch {
    std::vector<fd_operator *> ops;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    BatchPlan plan;
    int *status;
    cudaGraphExec_t graph;
    bool has_graph;
    int64_t graph_steps;
    int64_t launches;
};

static void batch_release(fd_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->has_graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    batch_plan_release(b->plan);
    if (b->status) cudaFree(b->status);
    delete b;
}

// (Re)build the batch for a tile height and depth: every shot's tiling, then
// the one device table of all shots.  Drops a captured graph (it holds the
// previous table).  On failure the batch has no plan until the next build.
static fd_status batch_build(fd_batch *b, int rows, int stages)
{
    if (b->has_graph) {
        cudaGraphExecDestroy(b->graph);
        b->has_graph = false;
    }
    batch_plan_release(b->plan);
    for (size_t i = 0; i < b->ops.size(); i++) {
        fd_operator *op = b->ops[i];
        fd_status s = fd_operator_set_tiling(op, rows, 0);
        if (s != FD_OK) return s;
        if (op->src && op->src->npoint > 0 && !op->tma.has_src)
            return set_error(FD_ERR_UNSUPPORTED, "fd_batch: operator %d's sources do not fit the tiles", (int)i);
    }
    std::vector<const TmaPlan *> plans;
    std::vector<const SparseDev *> recs;
    std::vector<float *> rtr;
    std::vector<long long> rst, sst;
    std::vector<const float *> str;
    for (fd_operator *op : b->ops) {
        plans.push_back(&op->tma);
        const bool hr = op->rec && op->rec->npoint > 0, hs = op->src && op->src->npoint > 0;
        recs.push_back(hr ? &op->rec->dev : nullptr);
        rtr.push_back(hr ? op->rec->trace : nullptr);
        rst.push_back(hr ? op->rec->stride : 0);
        str.push_back(hs ? op->src->trace : nullptr);
        sst.push_back(hs ? op->src->stride : 0);
    }
    return batch_plan_build(b->plan, plans, recs, rtr, rst, str, sst, b->ops[0]->coef, stages, b->stream);
}

extern "C" fd_status fd_batch_create(fd_operator *const *ops, int nops, int rows, int stages, fd_batch **out)
{
    if (!ops || nops < 1 || !out || rows < 0 || stages < 0)
        return set_error(FD_ERR_INVALID_ARG, "fd_batch_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < nops; i++) {
        fd_operator *op = ops[i];
        if (!op) return set_error(FD_ERR_INVALID_ARG, "fd_batch_create: null operator %d", i);
        if (op->kind != FD_ACOUSTIC_LEAPFROG || op->geom.ndim != 3 || !op->tma.ready)
            return set_error(FD_ERR_UNSUPPORTED, "fd_batch_create: operator %d is not a tiled 3D acoustic operator", i);
        if (op->flags & (FD_FLAG_REVERSE | FD_FLAG_PLAIN_KERNELS))
            return set_error(FD_ERR_UNSUPPORTED, "fd_batch_create: operator %d: forward tiled operators only", i);
        if (op->so != ops[0]->so || std::memcmp(&op->coef, &ops[0]->coef, sizeof(Coef)) != 0)
            return set_error(FD_ERR_UNSUPPORTED, "fd_batch_create: operators differ in space order or spacing");
        if (op->stream != ops[0]->stream)
            return set_error(FD_ERR_INVALID_ARG, "fd_batch_create: operators on different streams");
    }
    fd_batch *b = new (std::nothrow) fd_batch();
    if (!b) return set_error(FD_ERR_NOMEM, "fd_batch_create: out of host memory");
    b->ops.assign(ops, ops + nops);
    b->stream = ops[0]->stream;
    b->capture_stream = nullptr;
    b->status = nullptr;
    b->has_graph = false;
    b->graph_steps = 0;
    b->launches = 0;
    fd_status s = batch_build(b, rows > 0 ? rows : 16, stages > 0 ? stages : 3);
    if (s != FD_OK) {
        batch_release(b);
        return s;
    }
    cudaError_t e = cudaMalloc((void **)&b->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_release(b);
        return cuda_error(e, "fd_batch_create");
    }
    *out = b;
    return FD_OK;
}

// Validate a run of the batch and prepare every operator's coefficients.
static fd_status batch_prepare(fd_batch *b, int64_t t0, int64_t nt, double dt, const char *who)
{
    if (nt < 0 || t0 < 0) return set_error(FD_ERR_INVALID_ARG, "%s: need t0 >= 0, nt >= 0", who);
    for (fd_operator *op : b->ops) {
        for (fd_sparse *sp : {op->src, op->rec})
            if (sp && sp->npoint > 0 && t0 + nt > sp->nt)
                return set_error(FD_ERR_INVALID_ARG, "%s: a trace has %lld rows, need %lld", who, (long long)sp->nt,
                                 (long long)(t0 + nt));
        fd_status s = check_dt(op, dt, who);
        if (s != FD_OK) return s;
        s = prepare_coefficients(op, dt);
        if (s != FD_OK) return s;
    }
    return FD_OK;
}

static fd_status batch_enqueue(fd_batch *b, int64_t t0, int64_t nt, cudaStream_t st)
{
    for (int64_t n = t0; n < t0 + nt; n++) {
        FD_CUDA(launch_batch(b->plan, (long long)n, (int)(n & 1), b->status, st), "batch step");
        b->launches += 1;
    }
    return FD_OK;
}

extern "C" fd_status fd_batch_apply(fd_batch *b, int64_t t0, int64_t nt, double dt)
{
    if (!b) return set_error(FD_ERR_INVALID_ARG, "fd_batch_apply: null batch");
    fd_status s = batch_prepare(b, t0, nt, dt, "fd_batch_apply");
    if (s != FD_OK) return s;
    return batch_enqueue(b, t0, nt, b->stream);
}

extern "C" fd_status fd_batch_autotune(fd_batch *b, int64_t t0, int64_t nsteps, double dt, int *best_rows,
                                       int *best_stages, double *best_ms_per_step)
{
    if (!b || nsteps < 1 || t0 < 0) return set_error(FD_ERR_INVALID_ARG, "fd_batch_autotune: bad arguments");
    fd_status s = batch_prepare(b, t0, nsteps, dt, "fd_batch_autotune");
    if (s != FD_OK) return s;
    static const int kRows[] = {10, 12, 14, 16, 20, 24, 27, 30};
    cudaEvent_t e0, e1;
    FD_CUDA(cudaEventCreate(&e0), "fd_batch_autotune");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(FD_ERR_CUDA, "fd_batch_autotune: cudaEventCreate");
    }
    int br = 0, bs = 0;
    double bms = 1e30;
    fd_status last = FD_OK;
    for (int rows : kRows) {
        for (int stages = 2; stages <= 4 && last == FD_OK; stages++) {
            if (batch_build(b, rows, stages) != FD_OK) continue;  // does not fit: next candidate
            last = batch_enqueue(b, t0, nsteps < 3 ? nsteps : 3, b->stream);  // warm-up
            if (last != FD_OK) break;
            cudaEventRecord(e0, b->stream);
            last = batch_enqueue(b, t0, nsteps, b->stream);
            cudaEventRecord(e1, b->stream);
            if (last != FD_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                last = set_error(FD_ERR_CUDA, "fd_batch_autotune: timing");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double per = ms / (double)nsteps;
            if (per < bms) {
                bms = per;
                br = rows;
                bs = stages;
            }
        }
        if (last != FD_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (last != FD_OK) return last;
    if (br == 0) return set_error(FD_ERR_UNSUPPORTED, "fd_batch_autotune: no tiling fits");
    s = batch_build(b, br, bs);
    if (s != FD_OK) return s;
    // the trial runs may have written the status word: report it now
    FD_CUDA(cudaStreamSynchronize(b->stream), "fd_batch_autotune");
    int status = 0;
    FD_CUDA(cudaMemcpy(&status, b->status, sizeof status, cudaMemcpyDeviceToHost), "fd_batch_autotune: status");
    if (status != 0) {
        cudaMemset(b->status, 0, sizeof(int));
        return set_error(FD_ERR_TIMEOUT, "fd_batch_autotune: a device wait gave up (code %d)", status);
    }
    if (best_rows) *best_rows = br;
    if (best_stages) *best_stages = bs;
    if (best_ms_per_step) *best_ms_per_step = bms;
    return FD_OK;
}

extern "C" fd_status fd_batch_capture(fd_batch *b, int64_t t0, int64_t nt, double dt)
{
    if (!b || nt < 1) return set_error(FD_ERR_INVALID_ARG, "fd_batch_capture: bad arguments");
    fd_status s = batch_prepare(b, t0, nt, dt, "fd_batch_capture");
    if (s != FD_OK) return s;
    FD_CUDA(cudaStreamSynchronize(b->stream), "fd_batch_capture");
    if (b->has_graph) {
        cudaGraphExecDestroy(b->graph);
        b->has_graph = false;
    }
    FD_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "fd_batch_capture: begin");
    const int64_t before = b->launches;
    s = batch_enqueue(b, t0, nt, b->capture_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &graph);
    b->launches = before;  // captured launches run at replay
    if (s != FD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_error(e, "fd_batch_capture: end");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "fd_batch_capture: instantiate");
    b->has_graph = true;
    b->graph_steps = nt;
    return FD_OK;
}

extern "C" fd_status fd_batch_replay(fd_batch *b)
{
    if (!b || !b->has_graph) return set_error(FD_ERR_INVALID_ARG, "fd_batch_replay: nothing captured");
    FD_CUDA(cudaGraphLaunch(b->graph, b->stream), "fd_batch_replay");
    b->launches += b->graph_steps;
    return FD_OK;
}

extern "C" fd_status fd_batch_sync(fd_batch *b)
{
    if (!b) return set_error(FD_ERR_INVALID_ARG, "fd_batch_sync: null batch");
    FD_CUDA(cudaStreamSynchronize(b->stream), "fd_batch_sync");
    int status = 0;
    FD_CUDA(cudaMemcpy(&status, b->status, sizeof status, cudaMemcpyDeviceToHost), "fd_batch_sync: status");
    if (status != 0) {
        cudaMemset(b->status, 0, sizeof(int));
        cudaDeviceSynchronize();
        return set_error(FD_ERR_TIMEOUT, "fd_batch_sync: a device wait gave up (code %d)", status);
    }
    return FD_OK;
}

extern "C" fd_status fd_batch_info(const fd_batch *b, int *rows, int *stages, int *ctas, int64_t *launches)
{
    if (!b) return set_error(FD_ERR_INVALID_ARG, "fd_batch_info: null batch");
    if (rows) *rows = b->plan.rows_max;
    if (stages) *stages = b->plan.P;
    if (ctas) *ctas = b->plan.nctas;
    if (launches) *launches = b->launches;
    return FD_OK;
}

extern "C" void fd_batch_destroy(fd_batch *b) { batch_release(b); }
