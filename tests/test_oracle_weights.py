"""Pins of the oracle's finite-difference weights (CPU only).

The closed-form central weights and the general Taylor-moment solver of the
oracle are checked against: an exact rational Vandermonde solve (brute force
in Python fractions), textbook values, the moment conditions, and the stencils
the paper prints for its convection (Eq. 2dconvdiscr) and Laplace
(Eq. 2dlaplace_discr) examples.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_weights(deriv, offsets):
    """Exact rational solution of sum_j w_j x_j^k / k! = [k == deriv]."""
    n = len(offsets)
    A = [[Fraction(x) ** k / math.factorial(k) for x in offsets] + [Fraction(int(k == deriv))]
         for k in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col] / A[col][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return [A[j][n] / A[j][j] for j in range(n)]


@pytest.mark.parametrize("so", [2, 4, 6, 8, 10, 12, 14, 16])
def test_central2_matches_exact_rationals(orc, so):
    M = so // 2
    exact = exact_weights(2, list(range(-M, M + 1)))
    w = orc.weights_central2(so)
    for k in range(M + 1):
        ex = float(exact[M + k])
        assert exact[M + k] == exact[M - k]  # symmetry of the exact stencil
        assert abs(w[k] - ex) <= 2 * np.spacing(abs(ex)), (so, k, w[k], ex)


def test_central2_textbook_values(orc):
    # Standard central second-difference weights (Fornberg 1988, Table 1).
    assert list(orc.weights_central2(2)) == [-2.0, 1.0]
    np.testing.assert_allclose(orc.weights_central2(4), [-5 / 2, 4 / 3, -1 / 12], rtol=1e-15)
    np.testing.assert_allclose(orc.weights_central2(8),
                               [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560], rtol=1e-15)


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_central2_moment_conditions(orc, so):
    M = so // 2
    w = orc.weights_central2(so)
    full = np.concatenate([w[:0:-1], w])
    k = np.arange(-M, M + 1, dtype=np.float64)
    assert abs(full.sum()) < 1e-13
    np.testing.assert_allclose((full * k ** 2).sum(), 2.0, rtol=1e-13)
    for p in range(4, so + 1, 2):  # higher even moments vanish up to the order
        assert abs((full * k ** p).sum()) < 1e-9 * math.factorial(p)
    # the first moment not cancelled gives the leading truncation error
    assert abs((full * k ** (so + 2)).sum()) > 1e-3


@pytest.mark.parametrize("deriv,offsets", [
    (1, [-1, 0]), (1, [0, 1]), (2, [-1, 0, 1]), (1, [-2, -1, 0, 1, 2]),
    (2, [0, 1, 2, 3]), (3, [-2, -1, 0, 1, 2]), (1, [-0.5, 0.5]), (2, [-1.5, -0.5, 0.5, 1.5]),
])
def test_general_weights_exact(orc, deriv, offsets):
    exact = [float(x) for x in exact_weights(deriv, [Fraction(o) for o in offsets])]
    np.testing.assert_allclose(orc.weights(deriv, offsets), exact, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("so", [2, 4, 8, 16])
def test_general_solver_agrees_with_closed_form(orc, so):
    M = so // 2
    wg = orc.weights(2, list(range(-M, M + 1)))
    wc = orc.weights_central2(so)
    np.testing.assert_allclose(wg[M:], wc, rtol=1e-9, atol=1e-12)


def _golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(None, 1)
            rows[k] = v
    return rows


def test_convection_stencil_matches_paper(orc):
    """The printed convection equation and its solved stencil (c = 1)."""
    g = _golden("convection_stencil.txt")
    wt = orc.weights(1, [0, 1])     # u.dt, forward difference: (u(t+s) - u(t))/s
    wx = orc.weights(1, [-1, 0])    # u.dxl, backward difference: (u(x) - u(x-h))/h
    wy = orc.weights(1, [-1, 0])    # u.dyl
    for s, h in [(0.01, 0.05), (0.3, 1.7)]:
        env = {"s": s, "h": h}
        ev = lambda key: eval(g[key], {}, env)  # noqa: E731
        c = 1.0
        eq_fwd = wt[1] / s
        eq_ctr = wt[0] / s + c * wx[1] / h + c * wy[1] / h
        eq_xm = c * wx[0] / h
        eq_ym = c * wy[0] / h
        np.testing.assert_allclose([eq_fwd, eq_ctr, eq_xm, eq_ym],
                                   [ev("eq_forward"), ev("eq_center"), ev("eq_x_minus_h"),
                                    ev("eq_y_minus_h")], rtol=1e-12)
        # solve for u(t+s)
        np.testing.assert_allclose([-eq_ctr / eq_fwd, -eq_xm / eq_fwd, -eq_ym / eq_fwd],
                                   [ev("center"), ev("x_minus_h"), ev("y_minus_h")], rtol=1e-12)


def test_laplace_jacobi_matches_paper(orc):
    """Eq. 2dlaplace_discr from the SO2 central weights, dx != dy."""
    g = _golden("laplace_jacobi.txt")
    w = orc.weights_central2(2)
    for dx, dy in [(0.1, 0.1), (0.03, 0.07)]:
        # w1 (p_{i+1}+p_{i-1})/dx^2 + w1 (p_{j+1}+p_{j-1})/dy^2 + w0 (1/dx^2 + 1/dy^2) p_ij = 0
        ctr = w[0] * (1 / dx ** 2 + 1 / dy ** 2)
        cx = -w[1] / dx ** 2 / ctr
        cy = -w[1] / dy ** 2 / ctr
        env = {"dx": dx, "dy": dy}
        np.testing.assert_allclose([cx, cy], [eval(g["x_neighbours"].replace("^", "**"), {}, env),
                                              eval(g["y_neighbours"].replace("^", "**"), {}, env)], rtol=1e-12)


def test_bad_orders_rejected(orc):
    for so in (0, 1, 3, 18):
        with pytest.raises(RuntimeError):
            orc.weights_central2(so)
    with pytest.raises(RuntimeError):
        orc.weights(1, [0.0, 0.0])
