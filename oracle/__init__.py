"""CPU oracle for the explicit finite-difference method (arXiv 1707.03776).

TEST INFRASTRUCTURE ONLY.  This package is the independent, slow, literal
reference the CUDA path is checked against.  Only the test suite, the smoke
check (`__graft_entry__.smoke`) and the benchmark's CPU-baseline leg may import
it.  It shares no code with the product package and never imports it.

The arithmetic lives in `fd_oracle.c` (plain C loop nests, FP64 and FP32);
this module only marshals numpy arrays through ctypes.  Conventions:
  * fields are dense row-major numpy arrays of shape `shape` (2D or 3D), with
    no halo stored: values outside the grid are zero (zero Dirichlet halo);
  * `m`, `eta` (square slowness, damping) are FP32 inputs;
  * sparse coordinates are FP64 [npoint, ndim] in physical units;
  * traces are time-major [nt, npoint].
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        _LIB = ctypes.CDLL(path)
    return _LIB


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _real(precision):
    if precision == "f64":
        return np.float64, ctypes.c_double
    if precision == "f32":
        return np.float32, ctypes.c_float
    raise ValueError(precision)


def _grid_args(shape, spacing, origin=None):
    ndim = len(shape)
    if ndim not in (2, 3):
        raise ValueError("ndim must be 2 or 3")
    shp = np.ascontiguousarray(shape, dtype=np.int64)
    spc = np.ascontiguousarray(spacing, dtype=np.float64)
    org = np.ascontiguousarray(origin if origin is not None else [0.0] * ndim, dtype=np.float64)
    return ndim, shp, spc, org


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def _coords(coords, ndim):
    if coords is None:
        return 0, None
    c = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, ndim)
    return c.shape[0], c


# --------------------------------------------------------------------------
# Weights
# --------------------------------------------------------------------------

def weights_central2(space_order):
    """Closed-form central second-derivative weights w_0..w_M (M = SO/2)."""
    w = np.zeros(9, dtype=np.float64)
    _check(_lib().or_weights_central2(ctypes.c_int(space_order), _p(w, ctypes.c_double)),
           "weights_central2")
    return w[: space_order // 2 + 1].copy()


def weights(deriv, offsets):
    """Weights for derivative `deriv` at 0 from samples at `offsets` (grid units)."""
    off = np.ascontiguousarray(offsets, dtype=np.float64)
    w = np.zeros(off.size, dtype=np.float64)
    _check(_lib().or_weights(ctypes.c_int(deriv), ctypes.c_int(off.size), _p(off, ctypes.c_double),
                             _p(w, ctypes.c_double)), "weights")
    return w


# --------------------------------------------------------------------------
# Building blocks
# --------------------------------------------------------------------------

def laplacian(u, spacing, space_order, precision="f64"):
    dt_, ct = _real(precision)
    u = np.ascontiguousarray(u, dtype=dt_)
    ndim, shp, spc, _ = _grid_args(u.shape, spacing)
    out = np.empty_like(u)
    fn = getattr(_lib(), "or_laplacian_" + precision)
    _check(fn(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
              ctypes.c_int(space_order), _p(u, ct), _p(out, ct)), "laplacian")
    return out


def table(shape, spacing, origin, coords):
    """Interpolation table: (nodes [np, 2^ndim, ndim] int64, weights [np, 2^ndim])."""
    ndim, shp, spc, org = _grid_args(shape, spacing, origin)
    npnt, c = _coords(coords, ndim)
    nc = 1 << ndim
    nodes = np.zeros((npnt, nc, ndim), dtype=np.int64)
    w = np.zeros((npnt, nc), dtype=np.float64)
    _check(_lib().or_table(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
                           _p(org, ctypes.c_double), ctypes.c_int(npnt), _p(c, ctypes.c_double),
                           _p(nodes, ctypes.c_int64), _p(w, ctypes.c_double)), "table")
    return nodes, w


def interpolate(u, spacing, origin, coords, precision="f64"):
    dt_, ct = _real(precision)
    u = np.ascontiguousarray(u, dtype=dt_)
    ndim, shp, spc, org = _grid_args(u.shape, spacing, origin)
    npnt, c = _coords(coords, ndim)
    out = np.zeros(npnt, dtype=dt_)
    fn = getattr(_lib(), "or_interpolate_" + precision)
    _check(fn(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
              _p(org, ctypes.c_double), ctypes.c_int(npnt), _p(c, ctypes.c_double),
              _p(u, ct), _p(out, ct)), "interpolate")
    return out


def interpolate_from_f32(u32, spacing, origin, coords):
    """rec = R u in FP64 arithmetic from an FP32 field (for sampled checks)."""
    u = np.ascontiguousarray(u32, dtype=np.float32)
    ndim, shp, spc, org = _grid_args(u.shape, spacing, origin)
    npnt, c = _coords(coords, ndim)
    out = np.zeros(npnt, dtype=np.float64)
    _check(_lib().or_interpolate_from_f32(
        ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
        _p(org, ctypes.c_double), ctypes.c_int(npnt), _p(c, ctypes.c_double),
        _p(u, ctypes.c_float), _p(out, ctypes.c_double)), "interpolate_from_f32")
    return out


# --------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------

def acoustic_forward(shape, spacing, origin, space_order, m, eta, dt, nt,
                     src_coords=None, src_trace=None, rec_coords=None,
                     u_cur=None, u_prev=None, t0=0, n_total=None, precision="f64"):
    """Forward acoustic modelling for steps t0..t0+nt-1.

    Returns (u_cur, u_prev, rec_trace): the states u^{t0+nt}, u^{t0+nt-1} and
    the receiver trace [n_total, nrec] (rows t0..t0+nt-1 filled, others 0).
    """
    dt_, ct = _real(precision)
    ndim, shp, spc, org = _grid_args(shape, spacing, origin)
    shape = tuple(int(s) for s in shape)
    m = np.ascontiguousarray(m, dtype=np.float32).reshape(shape)
    eta_a = None if eta is None else np.ascontiguousarray(eta, dtype=np.float32).reshape(shape)
    uc = np.zeros(shape, dt_) if u_cur is None else np.array(u_cur, dtype=dt_, copy=True).reshape(shape)
    up = np.zeros(shape, dt_) if u_prev is None else np.array(u_prev, dtype=dt_, copy=True).reshape(shape)
    n_total = (t0 + nt) if n_total is None else n_total
    nsrc, sc = _coords(src_coords, ndim)
    nrec, rc_ = _coords(rec_coords, ndim)
    st = None
    if nsrc:
        st = np.ascontiguousarray(src_trace, dtype=dt_).reshape(n_total, nsrc)
    rt = np.zeros((n_total, max(nrec, 1)), dtype=dt_)
    fn = getattr(_lib(), "or_acoustic_forward_" + precision)
    rcode = fn(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
               _p(org, ctypes.c_double), ctypes.c_int(space_order),
               _p(m, ctypes.c_float), _p(eta_a, ctypes.c_float), ctypes.c_double(dt),
               ctypes.c_int64(t0), ctypes.c_int64(nt), _p(uc, ct), _p(up, ct),
               ctypes.c_int(nsrc), _p(sc, ctypes.c_double), _p(st, ct),
               ctypes.c_int(nrec), _p(rc_, ctypes.c_double), _p(rt, ct))
    _check(rcode, "acoustic_forward")
    return uc, up, rt[:, :nrec]


def acoustic_adjoint(shape, spacing, origin, space_order, m, eta, dt, nt,
                     rec_coords, rec_trace, src_coords, precision="f64"):
    """Adjoint modelling: returns (srca [nt, nsrc], mu^0 field)."""
    dt_, ct = _real(precision)
    ndim, shp, spc, org = _grid_args(shape, spacing, origin)
    shape = tuple(int(s) for s in shape)
    m = np.ascontiguousarray(m, dtype=np.float32).reshape(shape)
    eta_a = None if eta is None else np.ascontiguousarray(eta, dtype=np.float32).reshape(shape)
    nrec, rc_ = _coords(rec_coords, ndim)
    nsrc, sc = _coords(src_coords, ndim)
    rt = np.ascontiguousarray(rec_trace, dtype=dt_).reshape(nt, nrec)
    sa = np.zeros((nt, max(nsrc, 1)), dtype=dt_)
    mu = np.zeros(shape, dt_)
    fn = getattr(_lib(), "or_acoustic_adjoint_" + precision)
    rcode = fn(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
               _p(org, ctypes.c_double), ctypes.c_int(space_order),
               _p(m, ctypes.c_float), _p(eta_a, ctypes.c_float), ctypes.c_double(dt),
               ctypes.c_int64(nt), ctypes.c_int(nrec), _p(rc_, ctypes.c_double), _p(rt, ct),
               ctypes.c_int(nsrc), _p(sc, ctypes.c_double), _p(sa, ct), _p(mu, ct))
    _check(rcode, "acoustic_adjoint")
    return sa[:, :nsrc], mu


def diffusion(u0, spacing, space_order, a, dt, nt, precision="f64"):
    """Explicit Euler diffusion u <- u + a dt L u, nt steps; returns u^nt."""
    dt_, ct = _real(precision)
    u = np.array(u0, dtype=dt_, copy=True)
    ndim, shp, spc, _ = _grid_args(u.shape, spacing)
    fn = getattr(_lib(), "or_diffusion_" + precision)
    _check(fn(ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
              ctypes.c_int(space_order), ctypes.c_double(a), ctypes.c_double(dt),
              ctypes.c_int64(nt), _p(u, ct)), "diffusion")
    return u


def convection(u0, spacing, c, dt, nt, precision="f64"):
    """Linear convection (Eq. 2dconvdiscr), nt upwind steps on a 2D grid with
    the zero halo; returns u^nt."""
    dt_, ct = _real(precision)
    u = np.array(u0, dtype=dt_, copy=True)
    assert u.ndim == 2
    shp = np.array(u.shape, dtype=np.int64)
    spc = np.array(spacing, dtype=np.float64)
    fn = getattr(_lib(), "or_convection_" + precision)
    _check(fn(_p(shp, ctypes.c_int64), _p(spc, ctypes.c_double), ctypes.c_double(c), ctypes.c_double(dt),
              ctypes.c_int64(nt), _p(u, ct)), "convection")
    return u


def laplace(p0, spacing, tol, max_iter, precision="f64"):
    """Jacobi sweeps of the Laplace example (Eq. 2dlaplace_discr with its
    Dirichlet rows and Neumann columns); with tol > 0 until the L1 criterion
    r < tol.  Returns (p, sweeps done, last r)."""
    dt_, ct = _real(precision)
    p = np.array(p0, dtype=dt_, copy=True)
    assert p.ndim == 2
    shp = np.array(p.shape, dtype=np.int64)
    spc = np.array(spacing, dtype=np.float64)
    it = ctypes.c_int64(0)
    r = ctypes.c_double(0.0)
    fn = getattr(_lib(), "or_laplace_" + precision)
    _check(fn(_p(shp, ctypes.c_int64), _p(spc, ctypes.c_double), ctypes.c_double(tol), ctypes.c_int64(max_iter),
              _p(p, ct), ctypes.byref(it), ctypes.byref(r)), "laplace")
    return p, int(it.value), float(r.value)


def step_points(shape, spacing, space_order, m, eta, dt, u_cur32, u_prev32, flat_idx):
    """One forward update (no injection) in FP64 at flat indices, from FP32 states."""
    ndim, shp, spc, _ = _grid_args(shape, spacing)
    m = np.ascontiguousarray(m, dtype=np.float32)
    eta_a = None if eta is None else np.ascontiguousarray(eta, dtype=np.float32)
    uc = np.ascontiguousarray(u_cur32, dtype=np.float32)
    up = np.ascontiguousarray(u_prev32, dtype=np.float32)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.zeros(idx.size, dtype=np.float64)
    _check(_lib().or_step_points_f64(
        ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double),
        ctypes.c_int(space_order), _p(m, ctypes.c_float), _p(eta_a, ctypes.c_float),
        ctypes.c_double(dt), _p(uc, ctypes.c_float), _p(up, ctypes.c_float),
        ctypes.c_int64(idx.size), _p(idx, ctypes.c_int64), _p(out, ctypes.c_double)),
        "step_points")
    return out


_THREADS = None


def num_threads():
    """Threads the OpenMP loops of the oracle use (set_num_threads, else
    OMP_NUM_THREADS, else the cores)."""
    if _THREADS is not None:
        return _THREADS
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        try:
            return int(env)
        except ValueError:
            pass
    return os.cpu_count() or 1


def set_num_threads(n):
    """Threads for the oracle's later OpenMP loops (the OpenMP runtime's own
    omp_set_num_threads, reached through the loaded library); None restores
    the default."""
    global _THREADS
    fn = _lib().omp_set_num_threads
    fn.argtypes = [ctypes.c_int]
    fn.restype = None
    if n is None:
        _THREADS = None
        fn(ctypes.c_int(num_threads()))
    else:
        _THREADS = int(n)
        fn(ctypes.c_int(_THREADS))


def acoustic_gradient(shape, spacing, origin, space_order, m64, eta64, dt, nt, src_coords, src_trace,
                      rec_coords, d_obs, with_grad=True):
    """(J, dJ/dm) of J(m) = 1/2 sum (R u - d_obs)^2, FP64, m and eta in FP64."""
    ndim, shp, spc, org = _grid_args(shape, spacing, origin)
    shape = tuple(int(s) for s in shape)
    m = np.ascontiguousarray(m64, dtype=np.float64).reshape(shape)
    eta = None if eta64 is None else np.ascontiguousarray(eta64, dtype=np.float64).reshape(shape)
    nsrc, sc = _coords(src_coords, ndim)
    nrec, rc_ = _coords(rec_coords, ndim)
    st = np.ascontiguousarray(src_trace, dtype=np.float64).reshape(nt, nsrc)
    do = np.ascontiguousarray(d_obs, dtype=np.float64).reshape(nt, nrec)
    J = ctypes.c_double(0.0)
    g = np.zeros(shape, dtype=np.float64) if with_grad else None
    rcode = _lib().or_acoustic_gradient_f64(
        ctypes.c_int(ndim), _p(shp, ctypes.c_int64), _p(spc, ctypes.c_double), _p(org, ctypes.c_double),
        ctypes.c_int(space_order), _p(m, ctypes.c_double), _p(eta, ctypes.c_double), ctypes.c_double(dt),
        ctypes.c_int64(nt), ctypes.c_int(nsrc), _p(sc, ctypes.c_double), _p(st, ctypes.c_double),
        ctypes.c_int(nrec), _p(rc_, ctypes.c_double), _p(do, ctypes.c_double), ctypes.byref(J),
        _p(g, ctypes.c_double))
    _check(rcode, "acoustic_gradient")
    return J.value, g
