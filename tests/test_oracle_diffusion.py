"""Pins of the oracle's explicit diffusion (CPU only).

  * closed form: with zero Dirichlet nodes at 0 and n+1, the mode
    sin(k pi x) sin(l pi y) is an exact SO2 eigenvector, so u^n = lambda^n mode
    with lambda = 1 - 4 (a dt/h^2) (sin^2(k pi h/2) + sin^2(l pi h/2));
  * on the 256^2 ring workload (a dt/h^2 = 0.2) the update is a convex
    combination, so 0 <= u <= 1 (maximum principle), total heat decreases,
    and the ring's D4 symmetry about the centre is kept.
"""
import math

import numpy as np
import pytest

from paper_1707_03776_gb300 import workloads as wl


@pytest.mark.parametrize("k,l", [(1, 1), (3, 2), (7, 5)])
def test_eigenmode_closed_form(orc, k, l):
    n = 62  # interior nodes 1..62, Dirichlet nodes 0 and 63
    h = 1.0 / (n + 1)
    a = 0.5
    dt = 0.2 * h * h / a
    x = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    mode = np.sin(k * math.pi * X) * np.sin(l * math.pi * Y)
    lam = 1.0 - 4.0 * 0.2 * (math.sin(k * math.pi * h / 2) ** 2 + math.sin(l * math.pi * h / 2) ** 2)
    nt = 150
    u = orc.diffusion(mode, (h, h), 2, a, dt, nt)
    np.testing.assert_allclose(u, lam ** nt * mode, rtol=0, atol=1e-13)


def test_ring_maximum_principle_and_symmetry(orc):
    cfg = wl.diffusion_ring()
    u = orc.diffusion(cfg["u0"].astype(np.float64), cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"])
    assert u.min() >= 0.0 and u.max() <= 1.0
    assert u.sum() < cfg["u0"].astype(np.float64).sum()
    for t in (u.T, u[::-1, :], u[:, ::-1], u[::-1, ::-1].T):
        np.testing.assert_allclose(t, u, rtol=0, atol=1e-13)
    # heat has spread from the ring into its centre
    c = u.shape[0] // 2
    assert u[c, c] > 0.0


def test_fp32_agrees_with_fp64(orc):
    cfg = wl.diffusion_ring(n=96, nt=200)
    u64 = orc.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"])
    u32 = orc.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"], precision="f32")
    assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-6


def test_high_order_diffusion_polynomial(orc):
    """One step of u + a dt L u on a quartic reproduces the exact Laplacian
    (SO4 is exact for degree <= 5) away from the halo."""
    n = 20
    h = 0.1
    x = (np.arange(n) - n / 2) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    u0 = X ** 4 + X * Y ** 3
    a, dt = 0.3, 1e-3
    u1 = orc.diffusion(u0, (h, h), 4, a, dt, 1)
    exact = u0 + a * dt * (12 * X ** 2 + 6 * X * Y)
    np.testing.assert_allclose(u1[2:-2, 2:-2], exact[2:-2, 2:-2], rtol=0, atol=1e-12)
