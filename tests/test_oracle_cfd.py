"""Pins of the oracle's Linear Convection and Laplace operators (CPU only).

Convection (Eq. 2dconvdiscr):
  * one step equals the paper's printed solved stencil (golden
    convection_stencil.txt, evaluated for random h and s);
  * at Courant number 1 along x (and none along y) a step is an exact shift
    by one node, with zero inflow;
  * with nu_x + nu_y <= 1 the update is a convex combination: the maximum
    principle holds;
  * the sum over the grid changes only by the outflow through the last row
    and column (the upwind fluxes telescope).
Laplace (Eq. 2dlaplace_discr with its boundary expressions):
  * one sweep's interior equals the paper's printed rearrangement (golden
    laplace_jacobi.txt);
  * a field linear in x, constant in y, is a fixed point (the discrete
    solution for p = 0 and p = C on the two x rows);
  * the converged field equals the direct solve of the same discrete
    equations (numpy.linalg.solve), boundary expressions included;
  * the stopping rule stops at the first sweep whose r is below tol.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, expr = line.split(None, 1)
        out[key] = expr.replace("^", "**")
    return out


def test_convection_matches_printed_stencil():
    g = _golden("convection_stencil.txt")
    rng = np.random.default_rng(1)
    u = rng.standard_normal((9, 7))
    h, s = 0.05, 0.013
    coef = {k: eval(v, {"h": h, "s": s}) for k, v in g.items()}
    got = oracle.convection(u, (h, h), 1.0, s, 1)
    up = np.zeros((11, 9))
    up[1:-1, 1:-1] = u
    ref = coef["center"] * u + coef["x_minus_h"] * up[:-2, 1:-1] + coef["y_minus_h"] * up[1:-1, :-2]
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-14)


def test_convection_unit_courant_is_a_shift():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((8, 6))
    got = oracle.convection(u, (0.1, 1e300), 2.0, 0.05, 3)  # c dt / dx = 1
    ref = np.zeros_like(u)
    ref[3:] = u[:-3]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_convection_maximum_principle_and_outflow():
    rng = np.random.default_rng(3)
    u = rng.uniform(0.0, 2.0, (20, 17))
    hx, hy, c, dt = 0.1, 0.08, 1.0, 0.03  # nu_x + nu_y = 0.675
    v = oracle.convection(u, (hx, hy), c, dt, 40)
    assert v.min() >= 0.0 and v.max() <= 2.0 + 1e-12
    one = oracle.convection(u, (hx, hy), c, dt, 1)
    nux, nuy = c * dt / hx, c * dt / hy
    expect = u.sum() - nux * u[-1, :].sum() - nuy * u[:, -1].sum()
    assert abs(one.sum() - expect) < 1e-12 * abs(u).sum()


def test_laplace_sweep_matches_printed_rearrangement():
    g = _golden("laplace_jacobi.txt")
    rng = np.random.default_rng(4)
    p = rng.standard_normal((7, 9))
    dx, dy = 0.2, 0.125
    wx = eval(g["x_neighbours"], {"dx": dx, "dy": dy})
    wy = eval(g["y_neighbours"], {"dx": dx, "dy": dy})
    got, it, _ = oracle.laplace(p, (dx, dy), 0.0, 1)
    assert it == 1
    ref = wx * (p[2:, 1:-1] + p[:-2, 1:-1]) + wy * (p[1:-1, 2:] + p[1:-1, :-2])
    np.testing.assert_allclose(got[1:-1, 1:-1], ref, rtol=1e-13, atol=1e-14)
    # boundary expressions: the x rows keep their values except the corners,
    # which the Neumann copies (applied last) set from the next column
    np.testing.assert_array_equal(got[0, 1:-1], p[0, 1:-1])
    np.testing.assert_array_equal(got[-1, 1:-1], p[-1, 1:-1])
    np.testing.assert_array_equal(got[:, 0], got[:, 1])
    np.testing.assert_array_equal(got[:, -1], got[:, -2])


def test_laplace_linear_field_is_a_fixed_point():
    nx, ny = 12, 9
    x = np.arange(nx) / (nx - 1)
    p = np.repeat((2.5 * x)[:, None], ny, axis=1)
    got, _, _ = oracle.laplace(p, (0.3, 0.2), 0.0, 25)
    np.testing.assert_allclose(got, p, rtol=1e-14, atol=1e-14)


def _direct_solution(nx, ny, dx, dy, top, bottom):
    """The fixed point of the sweep (interior equations, Dirichlet rows,
    Neumann columns with the corners copied) as one linear system."""
    n = nx * ny
    A = np.zeros((n, n))
    b = np.zeros(n)
    wx = dy * dy / (2 * (dx * dx + dy * dy))
    wy = dx * dx / (2 * (dx * dx + dy * dy))
    idx = lambda i, j: i * ny + j  # noqa: E731
    for i in range(nx):
        for j in range(ny):
            k = idx(i, j)
            A[k, k] = 1.0
            if j == 0 or j == ny - 1:
                A[k, idx(i, 1 if j == 0 else ny - 2)] -= 1.0
            elif i == 0:
                b[k] = top[j]
            elif i == nx - 1:
                b[k] = bottom[j]
            else:
                for (di, dj), w in (((1, 0), wx), ((-1, 0), wx), ((0, 1), wy), ((0, -1), wy)):
                    A[k, idx(i + di, j + dj)] -= w
    return np.linalg.solve(A, b).reshape(nx, ny)


def test_laplace_converges_to_the_direct_solution():
    nx, ny = 14, 10
    dx, dy = 2.0 / (nx - 1), 1.0 / (ny - 1)
    y = np.arange(ny) * dy
    p = np.zeros((nx, ny))
    p[-1, :] = y  # p = y at x = 2, p = 0 at x = 0
    got, it, r = oracle.laplace(p, (dx, dy), 1e-15, 200000)
    assert r < 1e-15 and it < 200000
    ref = _direct_solution(nx, ny, dx, dy, np.zeros(ny), y)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)


def test_laplace_stopping_rule():
    nx, ny = 16, 11
    p = np.zeros((nx, ny))
    p[-1, :] = np.linspace(0.0, 1.0, ny)
    spacing = (2.0 / (nx - 1), 1.0 / (ny - 1))
    _, it, r = oracle.laplace(p, spacing, 1e-4, 100000)
    assert r < 1e-4 and it > 10
    _, it2, r2 = oracle.laplace(p, spacing, 0.0, it - 1)
    assert it2 == it - 1 and r2 >= 1e-4
    with pytest.raises(Exception):
        oracle.laplace(np.zeros((2, 5)), spacing, 1e-4, 10)
