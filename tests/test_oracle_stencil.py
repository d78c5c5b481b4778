"""Pins of the oracle's Laplacian and interpolation table (CPU only).

  * polynomial exactness of every space order up to its order, and failure
    one degree above it;
  * measured convergence order on smooth trigonometric fields;
  * brute force on a tiny 3D grid: the oracle's operator assembled column by
    column equals the Kronecker-sum matrix built from exact rational weights,
    and is symmetric negative definite;
  * the linear interpolation table reproduces (bi/tri)linear functions
    exactly, has non-negative weights summing to one and puts weight one on a
    node that a point sits on.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from test_oracle_weights import exact_weights


def coords(shape, spacing, shift):
    ax = [(np.arange(n) - s) * h for n, h, s in zip(shape, spacing, shift)]
    return np.meshgrid(*ax, indexing="ij")


def interior_mask(shape, M):
    mask = np.zeros(shape, dtype=bool)
    mask[tuple(slice(M, n - M) for n in shape)] = True
    return mask


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_polynomial_exactness(orc, so):
    M = so // 2
    shape = (2 * M + 5, 2 * M + 4, 2 * M + 6)
    spacing = (0.25, 0.3, 0.2)
    X, Y, Z = coords(shape, spacing, [n / 2.0 for n in shape])
    mask = interior_mask(shape, M)
    for axis, V in enumerate((X, Y, Z)):
        for p in range(0, so + 2):
            u = V ** p
            exact = p * (p - 1) * V ** (p - 2) if p >= 2 else np.zeros_like(V)
            Lu = orc.laplacian(u, spacing, so)
            # scale of the terms summed: |w| |u| / h^2
            w = np.abs(orc.weights_central2(so)).sum() * 2
            scale = w * np.abs(u).max() / spacing[axis] ** 2 + 1.0
            err = np.abs(Lu - exact)[mask].max()
            assert err <= 1e-12 * scale, (so, axis, p, err, scale)
        # degree so+2 is not reproduced: the order is exactly `so`
        p = so + 2
        u = V ** p
        exact = p * (p - 1) * V ** (p - 2)
        Lu = orc.laplacian(u, spacing, so)
        err = np.abs(Lu - exact)[mask].max()
        assert err > 1e-6 * np.abs(exact[mask]).max(), (so, axis, err)
    # a mixed monomial (exact since each axis sees a degree <= so polynomial)
    u = X ** 2 * Y ** 3 * Z
    exact = 2 * Y ** 3 * Z + 6 * X ** 2 * Y * Z
    Lu = orc.laplacian(u, spacing, so)
    assert np.abs(Lu - exact)[mask].max() < 1e-10


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_convergence_order(orc, so):
    """Error of L on sin(kx x) sin(ky y) at interior points falls like h^so."""
    kx, ky = 1.3, 0.7
    # choose kh so truncation dominates rounding at every level
    base = {2: 0.2, 4: 0.4, 8: 0.8, 16: 1.2}[so]
    errs = []
    hs = [base, base / 2, base / 4] if so < 16 else [0.8, 0.6, 0.45]
    M = so // 2
    for h in hs:
        L = 6.0  # domain length in each axis
        n = int(round(L / h)) + 2 * M + 1
        x = (np.arange(n) - n // 2) * h
        Xg, Yg = np.meshgrid(x, x, indexing="ij")
        u = np.sin(kx * Xg + 0.4) * np.sin(ky * Yg + 0.9)
        Lu = orc.laplacian(u, (h, h), so)
        exact = -(kx ** 2 + ky ** 2) * u
        c = n // 2  # the node at x = y = 0, the same physical point at every h
        errs.append(abs(Lu[c, c] - exact[c, c]))
    slopes = [math.log(errs[i] / errs[i + 1]) / math.log(hs[i] / hs[i + 1]) for i in range(len(hs) - 1)]
    for s in slopes:
        assert abs(s - so) < 0.35 * max(1, so / 4), (so, errs, slopes)


def dense_laplacian_exact(shape, spacing, so):
    """Kronecker-sum matrix of the zero-halo Laplacian from exact weights."""
    M = so // 2
    ex = exact_weights(2, list(range(-M, M + 1)))
    w = [float(x) for x in ex[M:]]
    mats = []
    for n in shape:
        D = np.zeros((n, n))
        for i in range(n):
            for k in range(-M, M + 1):
                j = i + k
                if 0 <= j < n:
                    D[i, j] = w[abs(k)]
        mats.append(D)
    N = int(np.prod(shape))
    L = np.zeros((N, N))
    for a, n in enumerate(shape):
        parts = [np.eye(m) for m in shape]
        parts[a] = mats[a] / spacing[a] ** 2
        K = parts[0]
        for P in parts[1:]:
            K = np.kron(K, P)
        L += K
    return L


@pytest.mark.parametrize("so,shape", [(2, (8, 8, 8)), (4, (8, 8, 8)), (8, (8, 8, 8)), (16, (5, 9, 7)),
                                      (4, (9, 11))])
def test_bruteforce_dense_operator(orc, so, shape):
    spacing = tuple(0.5 + 0.1 * a for a in range(len(shape)))
    N = int(np.prod(shape))
    Lo = np.zeros((N, N))
    e = np.zeros(N)
    for j in range(N):
        e[:] = 0.0
        e[j] = 1.0
        Lo[:, j] = orc.laplacian(e.reshape(shape), spacing, so).ravel()
    Ld = dense_laplacian_exact(shape, spacing, so)
    np.testing.assert_allclose(Lo, Ld, rtol=0, atol=1e-13 * np.abs(Ld).max())
    np.testing.assert_array_equal(Lo, Lo.T)
    ev = np.linalg.eigvalsh(Lo)
    assert ev.max() < 0.0


def test_laplacian_2d_is_3d_slab(orc):
    """A 2D field equals the middle plane of a 3D field constant in d0 whose
    d0 contribution is removed (checks the axis mapping of the 2D path)."""
    u2 = np.random.default_rng(3).standard_normal((11, 13))
    L2 = orc.laplacian(u2, (0.4, 0.7), 4)
    Ld = dense_laplacian_exact((11, 13), (0.4, 0.7), 4)
    np.testing.assert_allclose(L2.ravel(), Ld @ u2.ravel(), atol=1e-12)


# --------------------------------------------------------------------------
# Interpolation table
# --------------------------------------------------------------------------

@pytest.mark.parametrize("ndim", [2, 3])
def test_table_reproduces_multilinear(orc, ndim):
    shape = (7, 9, 6)[:ndim]
    spacing = (0.5, 1.25, 2.0)[:ndim]
    origin = (-1.0, 3.0, 0.5)[:ndim]
    g = np.random.default_rng(11)
    lo = np.array(origin)
    hi = lo + (np.array(shape) - 1) * np.array(spacing)
    pts = lo + (hi - lo) * g.random((200, ndim))
    pts[0] = hi  # upper corner exactly
    pts[1] = lo
    grids = np.meshgrid(*[origin[a] + np.arange(shape[a]) * spacing[a] for a in range(ndim)],
                        indexing="ij")
    # any function of the form prod_a (alpha_a + beta_a x_a) summed is reproduced
    coef = g.standard_normal((4, ndim, 2))
    f = np.zeros(shape)
    fx = np.zeros(len(pts))
    for t in range(4):
        term = np.ones(shape)
        tx = np.ones(len(pts))
        for a in range(ndim):
            term = term * (coef[t, a, 0] + coef[t, a, 1] * grids[a])
            tx = tx * (coef[t, a, 0] + coef[t, a, 1] * pts[:, a])
        f += term
        fx += tx
    out = orc.interpolate(f, spacing, origin, pts)
    np.testing.assert_allclose(out, fx, rtol=1e-12, atol=1e-12)
    nodes, w = orc.table(shape, spacing, origin, pts)
    assert (w >= 0).all()
    np.testing.assert_allclose(w.sum(axis=1), 1.0, rtol=0, atol=1e-15)
    assert (nodes >= 0).all() and (nodes < np.array(shape)).all()


def test_table_on_node_and_upper_face(orc):
    shape, spacing, origin = (5, 6, 7), (1.0, 2.0, 0.5), (0.0, 0.0, 0.0)
    pts = np.array([[2.0, 4.0, 1.5], [4.0, 10.0, 3.0], [0.0, 0.0, 0.0]])
    nodes, w = orc.table(shape, spacing, origin, pts)
    expect = [(2, 2, 3), (4, 5, 6), (0, 0, 0)]
    for p in range(3):
        hit = [tuple(nodes[p, c]) for c in range(8) if w[p, c] == 1.0]
        assert hit == [expect[p]]
        assert np.count_nonzero(w[p]) == 1
    with pytest.raises(RuntimeError):
        orc.table(shape, spacing, origin, np.array([[4.0001, 0.0, 0.0]]))
    with pytest.raises(RuntimeError):
        orc.table(shape, spacing, origin, np.array([[0.0, -1e-9, 0.0]]))
