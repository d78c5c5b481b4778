"""ctypes binding of libfdgb.so (include/fd.h): the same names as the C ABI,
argument marshalling only, plus thin objects named after the paper's API
(TimeData, DenseData, PointData, Operator; Design and API section) that own
torch device tensors laid out as fd_field_layout asks.

Every computation on grid data runs in the library's CUDA kernels.  There is
no CPU fallback: if libfdgb.so has not been built the first call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdgb.so")

FD_OK = 0
FD_ERR_INVALID_ARG = 1
FD_ERR_UNSUPPORTED = 2
FD_ERR_LAYOUT = 3
FD_ERR_OUT_OF_DOMAIN = 4
FD_ERR_UNSTABLE = 5
FD_ERR_CUDA = 6
FD_ERR_TIMEOUT = 7
FD_ERR_NOMEM = 8

FD_DIFFUSION_EULER = 1
FD_ACOUSTIC_LEAPFROG = 2
FD_CONVECTION_UPWIND = 3
FD_LAPLACE_JACOBI = 4

FD_FLAG_REVERSE = 1 << 0
FD_FLAG_NO_CFL_CHECK = 1 << 1
FD_FLAG_PLAIN_KERNELS = 1 << 2

_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_f64p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class FDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


class fd_op_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("space_order", ctypes.c_int),
                ("u", _vp), ("m", _vp), ("eta", _vp), ("a", ctypes.c_double),
                ("src", _vp), ("rec", _vp), ("cuda_stream", _vp), ("flags", ctypes.c_uint)]


_LIB = None

# (name, restype, argtypes) of every exported function
_SIGNATURES = [
    ("fd_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("fd_last_error", ctypes.c_char_p, []),
    ("fd_version", ctypes.c_int, []),
    ("fd_weights", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _c_f64p, _c_f64p]),
    ("fd_weights_central2", ctypes.c_int, [ctypes.c_int, _c_f64p]),
    ("fd_grid_create", ctypes.c_int, [ctypes.c_int, _c_i64p, _c_f64p, _c_f64p, ctypes.POINTER(_vp)]),
    ("fd_grid_destroy", None, [_vp]),
    ("fd_field_layout", ctypes.c_int, [_vp, ctypes.c_int, _c_i64p, _c_i64p, _c_i64p]),
    ("fd_field_wrap", ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_vp), _c_i64p, ctypes.POINTER(_vp)]),
    ("fd_field_destroy", None, [_vp]),
    ("fd_sparse_create", ctypes.c_int, [_vp, ctypes.c_int, _c_f64p, _vp, ctypes.c_int64, ctypes.c_int64, _vp,
                                        ctypes.POINTER(_vp)]),
    ("fd_sparse_set_trace", ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int64]),
    ("fd_sparse_destroy", None, [_vp]),
    ("fd_operator_create", ctypes.c_int, [ctypes.POINTER(fd_op_desc), ctypes.POINTER(_vp)]),
    ("fd_operator_bind", ctypes.c_int, [_vp, ctypes.c_char_p, _vp]),
    ("fd_operator_apply", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]),
    ("fd_operator_sync", ctypes.c_int, [_vp]),
    ("fd_operator_destroy", None, [_vp]),
    ("fd_operator_launch_count", ctypes.c_int64, [_vp]),
    ("fd_operator_profile", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("fd_operator_profile_read", ctypes.c_int, [_vp, _c_f64p, _c_i64p]),
    ("fd_interpolate_noalloc", ctypes.c_int, [_vp, ctypes.c_int, _c_f64p, _vp, _vp, _vp]),
    ("fd_operator_step", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, _vp, _vp, _vp]),
    ("fd_imaging_accumulate", ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("fd_imaging_accumulate_steps", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _vp]),
    ("fd_operator_apply_imaging", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, _vp, _vp,
                                                 _vp, _vp]),
    ("fd_operator_set_tiling", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    ("fd_operator_autotune", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _c_f64p]),
    ("fd_batch_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(_vp)]),
    ("fd_batch_apply", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]),
    ("fd_batch_autotune", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _c_f64p]),
    ("fd_batch_capture", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]),
    ("fd_batch_replay", ctypes.c_int, [_vp]),
    ("fd_batch_sync", ctypes.c_int, [_vp]),
    ("fd_batch_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), _c_i64p]),
    ("fd_batch_destroy", None, [_vp]),
    ("fd_cnn_pack_weights", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    ("fd_cnn_conv3d", ctypes.c_int, [_c_i64p, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int,
                                     _vp]),
    ("fd_cnn_pack_weights_tc", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    ("fd_cnn_conv3d_tc", ctypes.c_int, [_c_i64p, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int,
                                        _vp, _vp]),
    ("fd_cnn_conv3d_wgrad", ctypes.c_int, [_c_i64p, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
    ("fd_cnn_features_sub", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_uint64, _vp, _vp]),
    ("fd_cnn_features", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, _vp, _vp]),
    ("fd_cnn_restrict", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _vp, _vp]),
    ("fd_cnn_add_correction", ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _vp]),
    ("fd_cnn_mse_grad", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
    ("fd_cnn_adam", ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int64, _vp]),
    ("fd_operator_converge", ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    ("fd_operator_set_time_block", ctypes.c_int, [_vp, ctypes.c_int]),
    ("fd_operator_get_time_block", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("fd_operator_debug_stall", ctypes.c_int, [_vp, ctypes.c_int]),
    ("fd_operator_sources_fused", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    ("fd_operator_get_tiling", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
]

FD_NOALLOC_MAX_POINTS = 65536

EXPORTED = [s[0] for s in _SIGNATURES]


def lib():
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfdgb.so is missing (%s): build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _status_name(s):
    try:
        return lib().fd_status_string(int(s)).decode()
    except Exception:  # pragma: no cover - message formatting only
        return "status %d" % s


def _check(status):
    if status != FD_OK:
        raise FDError(status, lib().fd_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------
# C-ABI functions, same names
# --------------------------------------------------------------------------

def fd_status_string(status):
    return lib().fd_status_string(int(status)).decode()


def fd_last_error():
    return lib().fd_last_error().decode()


def fd_version():
    return lib().fd_version()


def fd_weights(deriv, offsets):
    off = _f64(offsets)
    w = np.zeros(off.size, dtype=np.float64)
    _check(lib().fd_weights(int(deriv), off.size, off.ctypes.data_as(_c_f64p), w.ctypes.data_as(_c_f64p)))
    return w


def fd_weights_central2(space_order):
    w = np.zeros(9, dtype=np.float64)
    _check(lib().fd_weights_central2(int(space_order), w.ctypes.data_as(_c_f64p)))
    return w[: space_order // 2 + 1].copy()


def fd_grid_create(shape, spacing, origin=None):
    shp = _i64(shape)
    spc = _f64(spacing)
    org = None if origin is None else _f64(origin)
    h = _vp()
    _check(lib().fd_grid_create(shp.size, shp.ctypes.data_as(_c_i64p), spc.ctypes.data_as(_c_f64p),
                                None if org is None else org.ctypes.data_as(_c_f64p), ctypes.byref(h)))
    return h


def fd_grid_destroy(h):
    lib().fd_grid_destroy(h)


def fd_field_layout(grid, space_order, ndim):
    padded = np.zeros(3, dtype=np.int64)
    strides = np.zeros(3, dtype=np.int64)
    off = ctypes.c_int64(0)
    _check(lib().fd_field_layout(grid, int(space_order), padded.ctypes.data_as(_c_i64p),
                                 strides.ctypes.data_as(_c_i64p), ctypes.byref(off)))
    return tuple(int(x) for x in padded[:ndim]), tuple(int(x) for x in strides[:ndim]), off.value


def fd_field_wrap(grid, dev_ptrs, strides=None):
    arr = (_vp * len(dev_ptrs))(*[int(p) for p in dev_ptrs])
    st = None if strides is None else _i64(strides)
    h = _vp()
    _check(lib().fd_field_wrap(grid, len(dev_ptrs), arr, None if st is None else st.ctypes.data_as(_c_i64p),
                               ctypes.byref(h)))
    return h


def fd_field_destroy(h):
    lib().fd_field_destroy(h)


def fd_sparse_create(grid, coords, dev_trace, nt, trace_stride, stream=0):
    c = _f64(coords)
    npoint = c.shape[0] if c.ndim > 1 else 0
    h = _vp()
    _check(lib().fd_sparse_create(grid, npoint, c.ctypes.data_as(_c_f64p) if npoint else None,
                                  int(dev_trace) or None, int(nt), int(trace_stride), int(stream) or None,
                                  ctypes.byref(h)))
    return h


def fd_sparse_set_trace(h, dev_trace, nt, trace_stride):
    _check(lib().fd_sparse_set_trace(h, int(dev_trace) or None, int(nt), int(trace_stride)))


def fd_sparse_destroy(h):
    lib().fd_sparse_destroy(h)


def fd_operator_create(kind, space_order, u, m=None, eta=None, a=0.0, src=None, rec=None, stream=0, flags=0):
    d = fd_op_desc(kind=kind, space_order=space_order, u=u, m=m, eta=eta, a=float(a), src=src, rec=rec,
                   cuda_stream=int(stream) or None, flags=flags)
    h = _vp()
    _check(lib().fd_operator_create(ctypes.byref(d), ctypes.byref(h)))
    return h


def fd_operator_bind(op, name, obj):
    if name == "a":
        v = ctypes.c_double(float(obj))
        _check(lib().fd_operator_bind(op, b"a", ctypes.cast(ctypes.byref(v), _vp)))
    else:
        _check(lib().fd_operator_bind(op, name.encode(), obj))


def fd_operator_apply(op, t0, nt, dt):
    _check(lib().fd_operator_apply(op, int(t0), int(nt), float(dt)))


def fd_operator_sync(op):
    _check(lib().fd_operator_sync(op))


def fd_operator_destroy(op):
    lib().fd_operator_destroy(op)


def fd_operator_launch_count(op):
    return int(lib().fd_operator_launch_count(op))


def fd_operator_profile(op, max_launches):
    _check(lib().fd_operator_profile(op, int(max_launches)))


def fd_operator_profile_read(op):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().fd_operator_profile_read(op, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def fd_operator_step(op, n, dt, u_cur, u_prev, u_next):
    """One out-of-place step between device buffers (data pointers)."""
    _check(lib().fd_operator_step(op, int(n), float(dt), int(u_cur), int(u_prev), int(u_next)))


def fd_imaging_accumulate(grid, scale, mu, u0, u1, u2, grad, stream=0):
    """grad += scale * mu * (u0 - 2 u1 + u2) (device pointers)."""
    _check(lib().fd_imaging_accumulate(grid, float(scale), int(mu), int(u0), int(u1), int(u2), int(grad),
                                       int(stream) or None))


def fd_imaging_accumulate_steps(grid, scale, mu, u, grad, stream=0):
    """The imaging of adjoint steps n, n-1, ..., n-k+1 in one pass: mu = k
    adjoint-state pointers (times n, n-1, ...), u = k + 2 forward-state
    pointers (times n, n-1, ...), device memory."""
    k = len(mu)
    if len(u) != k + 2:
        raise ValueError("need k + 2 forward states for k adjoint states")
    mu_arr = (ctypes.c_void_p * max(k, 1))(*[int(p) for p in mu])
    u_arr = (ctypes.c_void_p * len(u))(*[int(p) for p in u])
    _check(lib().fd_imaging_accumulate_steps(grid, float(scale), k, mu_arr, u_arr, int(grad), int(stream) or None))


def fd_operator_apply_imaging(op, n, dt, scale, u0, u1, u2, grad):
    """Step n of the operator with grad += scale * w * (u0 - 2 u1 + u2)
    accumulated from the field w the step writes (device pointers)."""
    _check(lib().fd_operator_apply_imaging(op, int(n), float(dt), float(scale), int(u0), int(u1), int(u2),
                                           int(grad)))


def fd_operator_set_tiling(op, rows=0, stages=0):
    _check(lib().fd_operator_set_tiling(op, int(rows), int(stages)))


def fd_operator_autotune(op, t0, nsteps, dt):
    """Time candidate tilings and keep the fastest: (rows, stages, ms per step)."""
    r, st, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().fd_operator_autotune(op, int(t0), int(nsteps), float(dt), ctypes.byref(r), ctypes.byref(st),
                                      ctypes.byref(ms)))
    return r.value, st.value, ms.value


def fd_operator_sources_fused(op):
    """True when the tiled sweep injects the operator's sources itself."""
    f = ctypes.c_int(0)
    _check(lib().fd_operator_sources_fused(op, ctypes.byref(f)))
    return bool(f.value)


def fd_operator_get_tiling(op):
    r, s, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().fd_operator_get_tiling(op, ctypes.byref(r), ctypes.byref(s), ctypes.byref(c)))
    return r.value, s.value, c.value


def fd_batch_create(op_handles, rows=0, stages=0):
    arr = (_vp * len(op_handles))(*[h.value if isinstance(h, _vp) else h for h in op_handles])
    h = _vp()
    _check(lib().fd_batch_create(arr, len(op_handles), int(rows), int(stages), ctypes.byref(h)))
    return h


def fd_batch_apply(b, t0, nt, dt):
    _check(lib().fd_batch_apply(b, int(t0), int(nt), float(dt)))


def fd_batch_autotune(b, t0, nsteps, dt):
    """Time candidate tilings of the batch and keep the fastest: (rows, stages, ms per step)."""
    r, st, ms = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(lib().fd_batch_autotune(b, int(t0), int(nsteps), float(dt), ctypes.byref(r), ctypes.byref(st),
                                   ctypes.byref(ms)))
    return r.value, st.value, ms.value


def fd_batch_capture(b, t0, nt, dt):
    _check(lib().fd_batch_capture(b, int(t0), int(nt), float(dt)))


def fd_batch_replay(b):
    _check(lib().fd_batch_replay(b))


def fd_batch_sync(b):
    _check(lib().fd_batch_sync(b))


def fd_batch_info(b):
    r, s, c, n = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int64(0)
    _check(lib().fd_batch_info(b, ctypes.byref(r), ctypes.byref(s), ctypes.byref(c), ctypes.byref(n)))
    return r.value, s.value, c.value, n.value


def fd_batch_destroy(b):
    lib().fd_batch_destroy(b)


def fd_operator_converge(op, t0, max_iter, tol):
    """Laplace convergence loop; returns (sweeps done, last r)."""
    it = ctypes.c_int64(0)
    r = ctypes.c_double(0.0)
    _check(lib().fd_operator_converge(op, int(t0), int(max_iter), float(tol), ctypes.byref(it), ctypes.byref(r)))
    return int(it.value), float(r.value)


def fd_operator_debug_stall(op, plane):
    _check(lib().fd_operator_debug_stall(op, int(plane)))


def fd_operator_set_time_block(op, k):
    _check(lib().fd_operator_set_time_block(op, int(k)))


def fd_operator_get_time_block(op):
    k = ctypes.c_int(0)
    n = ctypes.c_int(0)
    _check(lib().fd_operator_get_time_block(op, ctypes.byref(k), ctypes.byref(n)))
    return k.value, n.value


def _ptr(t):
    return None if t is None else (t if isinstance(t, int) else t.data_ptr())


def fd_cnn_pack_weights(w, cin, cout, flip, frag, stream=0):
    _check(lib().fd_cnn_pack_weights(_ptr(w), int(cin), int(cout), int(flip), _ptr(frag), int(stream) or None))


def fd_cnn_conv3d(shape, x, frag, bias, cout, relu, mask, y, y_fp32, stream=0):
    shp = _i64(shape)
    _check(lib().fd_cnn_conv3d(shp.ctypes.data_as(_c_i64p), _ptr(x), _ptr(frag), _ptr(bias), int(cout), int(relu),
                               _ptr(mask), _ptr(y), int(y_fp32), int(stream) or None))


def fd_cnn_pack_weights_tc(w, cin, cout, flip, frag, stream=0):
    _check(lib().fd_cnn_pack_weights_tc(_ptr(w), int(cin), int(cout), int(flip), _ptr(frag), int(stream) or None))


def fd_cnn_conv3d_tc(shape, x, frag, bias, cout, relu, mask, y, y_fp32, status, stream=0):
    shp = _i64(shape)
    _check(lib().fd_cnn_conv3d_tc(shp.ctypes.data_as(_c_i64p), _ptr(x), _ptr(frag), _ptr(bias), int(cout),
                                  int(relu), _ptr(mask), _ptr(y), int(y_fp32), _ptr(status), int(stream) or None))


def fd_cnn_conv3d_wgrad(shape, x, gy, cin, cout, gw, gb, stream=0):
    shp = _i64(shape)
    _check(lib().fd_cnn_conv3d_wgrad(shp.ctypes.data_as(_c_i64p), _ptr(x), _ptr(gy), int(cin), int(cout), _ptr(gw),
                                     _ptr(gb), int(stream) or None))


def fd_cnn_features(grid, u, u_prev, m, scale, vref, x, stream=0, noise=0.0, seed=0):
    _check(lib().fd_cnn_features(grid, _ptr(u), _ptr(u_prev), _ptr(m), float(scale), float(vref), float(noise),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, _ptr(x), int(stream) or None))


def fd_cnn_features_sub(grid, u, u_prev, m, sub, nsub, scale, vref, x, stream=0, noise=0.0, seed=0):
    """Closure features with nsub model descriptors (sub: nsub slots one after
    another)."""
    _check(lib().fd_cnn_features_sub(grid, _ptr(u), _ptr(u_prev), _ptr(m), _ptr(sub) if nsub else None, int(nsub),
                                     float(scale), float(vref), float(noise), int(seed) & (2 ** 64 - 1), _ptr(x),
                                     int(stream) or None))


def fd_cnn_restrict(fine_grid, fine, coarse_grid, coarse, factor, sumsq=None, stream=0):
    _check(lib().fd_cnn_restrict(fine_grid, _ptr(fine), coarse_grid, _ptr(coarse), int(factor), _ptr(sumsq),
                                 int(stream) or None))


def fd_cnn_add_correction(grid, u, corr, scale, stream=0):
    _check(lib().fd_cnn_add_correction(grid, _ptr(u), _ptr(corr), float(scale), int(stream) or None))


def fd_cnn_mse_grad(grid, pred, target, base, scale, gy, loss, stream=0):
    _check(lib().fd_cnn_mse_grad(grid, _ptr(pred), _ptr(target), _ptr(base), float(scale), _ptr(gy), _ptr(loss),
                                 int(stream) or None))


def fd_cnn_adam(params, grads, m1, m2, n, lr, beta1, beta2, eps, step, stream=0):
    _check(lib().fd_cnn_adam(_ptr(params), _ptr(grads), _ptr(m1), _ptr(m2), int(n), float(lr), float(beta1),
                             float(beta2), float(eps), int(step), int(stream) or None))


def fd_interpolate_noalloc(grid, coords, dev_field, dev_out, stream=0):
    """Interpolate a device field slot at host coordinates into dev_out
    without any allocation.  With coords None (no points) the call only does
    the per-device set-up: the first call on a device allocates the static
    table there, so make that call at start-up."""
    c = _f64(coords if coords is not None else np.zeros((0, 3)))
    npoint = c.shape[0] if c.ndim > 1 else 0
    _check(lib().fd_interpolate_noalloc(grid, npoint, c.ctypes.data_as(_c_f64p) if npoint else None,
                                        int(dev_field) or None, int(dev_out) or None, int(stream) or None))


# --------------------------------------------------------------------------
# Objects after the paper's API
# --------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream_handle(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Grid:
    """A regular grid: shape, spacing, origin (physical units)."""

    def __init__(self, shape, spacing, origin=None):
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.spacing = tuple(float(h) for h in spacing)
        self.origin = tuple(float(o) for o in (origin if origin is not None else [0.0] * self.ndim))
        self.handle = fd_grid_create(self.shape, self.spacing, self.origin)
        self.padded_shape, self.strides, _ = fd_field_layout(self.handle, 2, self.ndim)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            fd_grid_destroy(self.handle)
            self.handle = None


class _Field:
    levels = 1

    def __init__(self, name, grid, device="cuda"):
        torch = _torch()
        self.name = name
        self.grid = grid
        self.slots = [torch.zeros(grid.padded_shape, dtype=torch.float32, device=device)
                      for _ in range(self.levels)]
        self.handle = fd_field_wrap(grid.handle, [t.data_ptr() for t in self.slots], grid.strides)

    def view(self, level=0):
        """Interior view of one slot (shape = grid.shape)."""
        t = self.slots[level]
        return t[..., : self.grid.shape[-1]]

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            fd_field_destroy(self.handle)
            self.handle = None


class DenseData(_Field):
    """Static field (the paper's DenseData): one slot, e.g. m or eta."""
    levels = 1

    @property
    def data(self):
        return self.view(0)


class TimeData(_Field):
    """Time-dependent field with 2 slots: slot n % 2 holds time n."""
    levels = 2

    def at(self, n):
        return self.view(int(n) % 2)


class PointData:
    """Sparse off-grid points (the paper's PointData) with a device trace
    data[nt, npoint] (time-major)."""

    def __init__(self, name, grid, coords, nt, device="cuda", stream=None):
        torch = _torch()
        self.name = name
        self.grid = grid
        self.coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, grid.ndim)
        self.npoint = self.coords.shape[0]
        self.nt = int(nt)
        self.data = torch.zeros((self.nt, max(self.npoint, 1)), dtype=torch.float32, device=device)
        self.handle = fd_sparse_create(grid.handle, self.coords, self.data.data_ptr(), self.nt,
                                       self.data.stride(0), _stream_handle(stream))

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            fd_sparse_destroy(self.handle)
            self.handle = None


class Batch:
    """Many forward operators (shots) advanced with one launch per step."""

    def __init__(self, operators, rows=0, stages=0):
        self._ops = list(operators)
        self.handle = fd_batch_create([o.handle for o in self._ops], rows, stages)

    def apply(self, t0, nt, dt):
        fd_batch_apply(self.handle, t0, nt, dt)

    def autotune(self, t0, nsteps, dt):
        """Pick the fastest tiling on the batch's own data: (rows, stages,
        ms per step).  The trial runs advance the shots' fields."""
        return fd_batch_autotune(self.handle, t0, nsteps, dt)

    def capture(self, t0, nt, dt):
        fd_batch_capture(self.handle, t0, nt, dt)

    def replay(self):
        fd_batch_replay(self.handle)

    def sync(self):
        fd_batch_sync(self.handle)

    def info(self):
        return fd_batch_info(self.handle)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            fd_batch_destroy(self.handle)
            self.handle = None


class Operator:
    """An FD operator (the paper's Operator) applied for nt steps with `apply`."""

    def __init__(self, kind, space_order, u, m=None, eta=None, a=0.0, src=None, rec=None, stream=None,
                 flags=0):
        self.kind = kind
        self.space_order = space_order
        self._keep = [u, m, eta, src, rec]
        self.handle = fd_operator_create(kind, space_order, u.handle, m.handle if m else None,
                                         eta.handle if eta else None, a, src.handle if src else None,
                                         rec.handle if rec else None, _stream_handle(stream), flags)

    def bind(self, name, obj):
        if name in ("a",):
            fd_operator_bind(self.handle, name, obj)
        elif name == "stream":
            fd_operator_bind(self.handle, name, _stream_handle(obj))
        else:
            fd_operator_bind(self.handle, name, obj.handle if obj is not None else None)
            self._keep.append(obj)

    def apply(self, t0, nt, dt):
        fd_operator_apply(self.handle, t0, nt, dt)

    def sync(self):
        fd_operator_sync(self.handle)

    def converge(self, t0, max_iter, tol):
        """The Laplace example's convergence loop: (sweeps done, last r)."""
        return fd_operator_converge(self.handle, t0, max_iter, tol)

    @property
    def launches(self):
        return fd_operator_launch_count(self.handle)

    def profile(self, max_launches):
        fd_operator_profile(self.handle, max_launches)

    def profile_read(self):
        """(summed ms, launches) of the profiled grid-update kernel launches."""
        return fd_operator_profile_read(self.handle)

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            fd_operator_destroy(self.handle)
            self.handle = None
