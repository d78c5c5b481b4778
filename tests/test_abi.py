"""The C-ABI library loads on a machine without a GPU and exports every
function include/fd.h declares; host-only calls (weights, grids, layouts,
argument checks) behave as documented.  No kernel is launched here."""
import ctypes
import os
import re
from fractions import Fraction

import numpy as np
import pytest

from paper_1707_03776_gb300 import fd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(fd.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return fd.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(fd.EXPORTED)


def test_weights_exact(L):
    from test_oracle_weights import exact_weights
    for so in (2, 4, 8, 12, 16):
        M = so // 2
        ex = exact_weights(2, list(range(-M, M + 1)))
        w = fd.fd_weights_central2(so)
        # Fornberg's recurrence rounds a little more than the closed form: a
        # few ulp, far below the FP32 rounding the kernels apply afterwards
        np.testing.assert_allclose(w, [float(x) for x in ex[M:]], rtol=2e-14, atol=0)
    for deriv, off in [(1, [-1, 0]), (1, [0, 1]), (2, [-1, 0, 1]), (3, [-2, -1, 0, 1, 2]), (1, [-0.5, 0.5, 1.5])]:
        ex = [float(x) for x in exact_weights(deriv, [Fraction(o) for o in off])]
        np.testing.assert_allclose(fd.fd_weights(deriv, off), ex, rtol=1e-12, atol=1e-12)


def test_weight_errors(L):
    for so in (0, 3, 18):
        with pytest.raises(fd.FDError) as e:
            fd.fd_weights_central2(so)
        assert e.value.status == fd.FD_ERR_UNSUPPORTED
    with pytest.raises(fd.FDError) as e:
        fd.fd_weights(1, [0.0, 0.0])
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FDError):
        fd.fd_weights(2, [0.0, 1.0])


def test_grid_and_layout(L):
    g = fd.fd_grid_create((13, 17, 9), (1.0, 2.0, 3.0))
    padded, strides, off = fd.fd_field_layout(g, 8, 3)
    assert padded == (13, 17, 16) and strides == (17 * 16, 16, 1) and off == 0
    fd.fd_grid_destroy(g)
    g = fd.fd_grid_create((512, 512, 512), (10.0,) * 3)
    padded, strides, _ = fd.fd_field_layout(g, 8, 3)
    assert padded == (512, 512, 512)
    fd.fd_grid_destroy(g)
    g = fd.fd_grid_create((254, 254), (1 / 255, 1 / 255), (1 / 255, 1 / 255))
    assert fd.fd_field_layout(g, 2, 2)[0] == (254, 256)
    with pytest.raises(fd.FDError):
        fd.fd_field_layout(g, 5, 2)
    fd.fd_grid_destroy(g)
    for bad in [((1, 4, 4), (1.0,) * 3), ((4, 4, 4), (1.0, 0.0, 1.0)), ((4,), (1.0,))]:
        with pytest.raises(fd.FDError) as e:
            fd.fd_grid_create(*bad)
        assert e.value.status == fd.FD_ERR_INVALID_ARG


def test_wrap_checks_layout(L):
    g = fd.fd_grid_create((8, 9, 10), (1.0,) * 3)
    with pytest.raises(fd.FDError) as e:
        fd.fd_field_wrap(g, [4096, 8192], strides=(9 * 10, 10, 1))
    assert e.value.status == fd.FD_ERR_LAYOUT
    with pytest.raises(fd.FDError) as e:
        fd.fd_field_wrap(g, [4096 + 4, 8192])
    assert e.value.status == fd.FD_ERR_LAYOUT
    with pytest.raises(fd.FDError) as e:
        fd.fd_field_wrap(g, [4096, 4096])
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    h = fd.fd_field_wrap(g, [4096, 8192], strides=(9 * 16, 16, 1))
    fd.fd_field_destroy(h)
    fd.fd_grid_destroy(g)


def test_operator_argument_checks(L):
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_create(fd.FD_ACOUSTIC_LEAPFROG, 8, None)
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    g = fd.fd_grid_create((8, 9, 10), (1.0,) * 3)
    u = fd.fd_field_wrap(g, [4096, 8192])
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_create(99, 8, u)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_create(fd.FD_ACOUSTIC_LEAPFROG, 8, u)  # no m
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_create(fd.FD_DIFFUSION_EULER, 2, u, a=-1.0)
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_create(fd.FD_DIFFUSION_EULER, 2, u, a=1.0, flags=fd.FD_FLAG_REVERSE)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
    assert "reverse" in fd.fd_last_error()
    fd.fd_field_destroy(u)
    fd.fd_grid_destroy(g)


def test_sparse_domain_check_before_device(L):
    g = fd.fd_grid_create((8, 9, 10), (2.0, 2.0, 2.0), (1.0, 1.0, 1.0))
    with pytest.raises(fd.FDError) as e:
        fd.fd_sparse_create(g, np.array([[0.5, 2.0, 2.0]]), 4096, 10, 1)
    assert e.value.status == fd.FD_ERR_OUT_OF_DOMAIN
    with pytest.raises(fd.FDError) as e:
        fd.fd_sparse_create(g, np.array([[2.0, 2.0, 2.0]]), 4096, 10, 0)
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    fd.fd_grid_destroy(g)
    # grids need 2 nodes per axis (an axis of one node has no interpolation
    # cell and no stencil)
    with pytest.raises(fd.FDError) as e:
        fd.fd_grid_create((8, 1, 10), (2.0, 2.0, 2.0), (0.0, 0.0, 0.0))
    assert e.value.status == fd.FD_ERR_INVALID_ARG


def test_imaging_steps_argument_checks(L):
    """fd_imaging_accumulate_steps rejects a group size outside 1..4, null and
    misaligned buffers and a gradient that aliases an input before it
    launches anything (the pointers here are never dereferenced)."""
    g = fd.fd_grid_create((8, 9, 10), (1.0,) * 3)
    mu = [4096 * (i + 1) for i in range(4)]
    u = [65536 * (i + 1) for i in range(6)]
    grad = 1 << 24
    cases = [
        (([], u[:2], grad), fd.FD_ERR_INVALID_ARG),                      # k = 0
        (([4096] * 5, [8192] * 7, grad), fd.FD_ERR_INVALID_ARG),         # k = 5
        ((mu[:2], u[:4], 0), fd.FD_ERR_INVALID_ARG),                     # null grad
        (([mu[0], 0], u[:4], grad), fd.FD_ERR_INVALID_ARG),              # null adjoint state
        ((mu[:2], u[:3] + [0], grad), fd.FD_ERR_INVALID_ARG),            # null forward state
        ((mu[:2], [u[0] + 4] + u[1:4], grad), fd.FD_ERR_LAYOUT),         # misaligned input
        ((mu[:2], u[:4], grad + 8), fd.FD_ERR_LAYOUT),                   # misaligned grad
        ((mu[:2], u[:4], u[3]), fd.FD_ERR_INVALID_ARG),                  # grad aliases an input
    ]
    for (m_, u_, gr), status in cases:
        k = len(m_)
        mu_arr = (ctypes.c_void_p * max(k, 1))(*m_)
        u_arr = (ctypes.c_void_p * len(u_))(*u_)
        rc = L.fd_imaging_accumulate_steps(g, -1.0, k, mu_arr, u_arr, gr, None)
        assert rc == status, (k, rc, status, fd.fd_last_error())
    with pytest.raises(ValueError):
        fd.fd_imaging_accumulate_steps(g, -1.0, mu[:2], u[:3], grad)
    fd.fd_grid_destroy(g)
