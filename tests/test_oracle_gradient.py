"""Pins of the oracle's adjoint-state gradient (CPU only).

J(m) = 1/2 sum_n sum_r (R u^n - d)^2 for the forward operator started from
rest.  The gradient the oracle returns must match central finite differences
of J itself (FP64, O(eps^2) truncation) in random directions, in 2D and 3D,
with the sponge on; perturbing m where no wave ever reaches (a far corner on
a short run) must leave J unchanged, so the gradient must vanish there.
"""
import numpy as np
import pytest

from paper_1707_03776_gb300 import workloads as wl


def _case(ndim, so, n, nt, seed):
    shape = (n + 2, n, n + 1)[:ndim]
    h = (10.0,) * ndim
    origin = (0.0,) * ndim
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    g = np.random.default_rng(seed)
    m_true = 1.0 / v ** 2
    m0 = m_true * (1.0 + 0.05 * g.standard_normal(shape))  # a perturbed starting model
    sig = wl.sponge_sigma(shape, h, 3, 2500.0, ref_width=40)
    eta = m_true * sig
    dt = 0.35 * 10.0 / 2700.0
    src_c = wl.random_points(shape, h, origin, 2, seed, margin=2.0)
    rec_c = wl.random_points(shape, h, origin, 6, seed + 1, margin=1.0)
    src = np.stack([wl.ricker(nt, dt, 25.0), 0.5 * wl.ricker(nt, dt, 20.0)], axis=1)
    return shape, h, origin, m_true, m0, eta, dt, src_c, rec_c, src


@pytest.mark.parametrize("ndim,so,n,nt", [(2, 4, 20, 90), (3, 8, 11, 50), (3, 2, 9, 40)])
def test_gradient_matches_central_differences(orc, ndim, so, n, nt):
    shape, h, origin, m_true, m0, eta, dt, src_c, rec_c, src = _case(ndim, so, n, nt, 7 * n)
    # observed data from the true model
    _, _, d_obs = orc.acoustic_forward(shape, h, origin, so, m_true.astype(np.float32), None, dt, nt,
                                       src_coords=src_c, src_trace=src, rec_coords=rec_c)
    d_obs = d_obs.astype(np.float64)
    J0, grad = orc.acoustic_gradient(shape, h, origin, so, m0, eta, dt, nt, src_c, src, rec_c, d_obs)
    assert J0 > 0 and np.abs(grad).max() > 0
    g = np.random.default_rng(n)
    for _ in range(3):
        dm = g.standard_normal(shape) * m0
        eps = 1e-5
        Jp, _ = orc.acoustic_gradient(shape, h, origin, so, m0 + eps * dm, eta, dt, nt, src_c, src, rec_c, d_obs,
                                      with_grad=False)
        Jm, _ = orc.acoustic_gradient(shape, h, origin, so, m0 - eps * dm, eta, dt, nt, src_c, src, rec_c, d_obs,
                                      with_grad=False)
        fd = (Jp - Jm) / (2 * eps)
        an = float((grad * dm).sum())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_gradient_vanishes_outside_the_domain_of_dependence(orc):
    shape, h, origin, m_true, m0, eta, dt, src_c, rec_c, src = _case(3, 4, 16, 8, 3)
    src_c = np.array([[20.0, 20.0, 20.0]])
    rec_c = np.array([[30.0, 20.0, 20.0]])
    src = src[:, :1] + 1.0
    d_obs = np.zeros((8, 1))
    J0, grad = orc.acoustic_gradient(shape, h, origin, 4, m0, None, dt, 8, src_c, src, rec_c, d_obs)
    assert J0 > 0
    # 8 steps of an SO4 stencil reach 2*8 cells: the far corner is untouched
    assert np.abs(grad[-2:, -2:, -2:]).max() == 0.0
    assert np.abs(grad[:5, :5, :5]).max() > 0.0
