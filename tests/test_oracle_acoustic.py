"""Pins of the oracle's acoustic forward and adjoint operators (CPU only).

What fixes each part without trusting the oracle itself:
  * standing wave: with constant m and no damping, a Fourier mode evolves as
    cos(n theta) with cos(theta) = 1 - v^2 dt^2 / 2 * sum_a sigma_h(k_a) (the
    discrete dispersion relation, sigma_h from exact rational weights), exactly
    up to rounding inside the boundary's domain of dependence;
  * temporal order 2 against the semi-discrete solution (SO2 Dirichlet modes
    are exact eigenvectors of the truncated Laplacian);
  * damping: closed-form solution of the modal recurrence of
    m u_tt + eta u_t - lap u = 0, and its decay rate against exp(-eta t / 2m);
  * discrete energy conservation with damping off, monotone decay with it on;
  * injection of src*dt^2/m at an on-node point (the paper's source term);
  * the adjoint dot-product test (Seismic Inversion Example), 2D and 3D, and
    the adjoint compared with the explicit transpose of the assembled forward
    matrix on a tiny grid;
  * resuming from any step reproduces an uninterrupted run bit for bit;
  * FP32 loop nest agrees with the FP64 one to FP32 rounding.
"""
import math

import numpy as np
import pytest

from test_oracle_weights import exact_weights
from paper_1707_03776_gb300 import workloads as wl


def sigma_h(k, h, so):
    """Symbol of the exact-weight central 2nd difference: -(w0 + 2 sum w_j cos(jkh))/h^2."""
    M = so // 2
    w = [float(x) for x in exact_weights(2, list(range(-M, M + 1)))[M:]]
    return -(w[0] + 2 * sum(w[j] * math.cos(j * k * h) for j in range(1, M + 1))) / h ** 2


@pytest.mark.parametrize("so,nsteps", [(16, 2), (4, 7), (8, 3)])
def test_standing_wave_exact(orc, so, nsteps):
    M = so // 2
    n = 2 * nsteps * M + 12
    shape = (n, n + 2, n - 1)
    h = (10.0, 12.0, 8.0)
    k = (0.9 / h[0], 0.5 / h[1], 0.7 / h[2])
    v = 2000.0
    dt = 0.35 * min(h) / v
    m = np.full(shape, 1.0 / v ** 2, dtype=np.float32)
    vv = 1.0 / float(m.flat[0])  # v^2 as the FP32 m represents it
    grids = np.meshgrid(*[np.arange(shape[a]) * h[a] for a in range(3)], indexing="ij")
    mode = np.ones(shape)
    for a in range(3):
        mode *= np.sin(k[a] * grids[a] + 0.3 * (a + 1))
    cos_th = 1.0 - 0.5 * vv * dt ** 2 * sum(sigma_h(k[a], h[a], so) for a in range(3))
    th = math.acos(cos_th)
    u_cur, u_prev, _ = orc.acoustic_forward(shape, h, (0, 0, 0), so, m, None, dt, nsteps,
                                            u_cur=mode, u_prev=math.cos(th) * mode)
    expect = math.cos(nsteps * th) * mode
    r = nsteps * M
    sl = tuple(slice(r, s - r) for s in shape)
    np.testing.assert_allclose(u_cur[sl], expect[sl], rtol=0, atol=1e-12)
    # outside the domain of dependence the zero halo has already acted
    assert np.abs(u_cur - expect).max() > 1e-6


def dirichlet_mode(shape, p):
    """sin(pi p_a (i+1)/(n_a+1)) products: exact SO2 eigenvectors with zero halo."""
    mode = np.ones(shape)
    lam = 0.0
    for a, n in enumerate(shape):
        i = np.arange(n)
        sh = [1] * len(shape)
        sh[a] = n
        mode = mode * np.sin(math.pi * p[a] * (i + 1) / (n + 1)).reshape(sh)
    return mode


def test_temporal_order_two(orc):
    """Leapfrog error at fixed T against cos(omega_h t), omega_h^2 = v^2 lambda_h."""
    shape = (24, 20)
    h = (5.0, 5.0)
    v = 1500.0
    p = (2, 3)
    mode = dirichlet_mode(shape, p)
    lam = sum(4.0 / h[a] ** 2 * math.sin(math.pi * p[a] / (2 * (shape[a] + 1))) ** 2 for a in range(2))
    m = np.full(shape, 1.0 / v ** 2, dtype=np.float32)
    vv = 1.0 / float(m.flat[0])
    om = math.sqrt(vv * lam)
    T = 0.02
    errs = []
    dts = []
    for nsteps in (40, 80, 160):
        dt = T / nsteps
        # start exactly on the semi-discrete solution: u^0 = mode, u^{-1} = cos(om dt) mode
        u, _, _ = orc.acoustic_forward(shape, h, (0, 0), 2, m, None, dt, nsteps,
                                       u_cur=mode, u_prev=math.cos(om * dt) * mode)
        errs.append(np.abs(u - math.cos(om * T) * mode).max())
        dts.append(dt)
    slopes = [math.log(errs[i] / errs[i + 1]) / math.log(dts[i] / dts[i + 1]) for i in range(2)]
    for s in slopes:
        assert abs(s - 2.0) < 0.1, (errs, slopes)


def test_damped_mode_closed_form(orc):
    shape = (14, 11, 9)
    h = (10.0, 10.0, 10.0)
    v = 1800.0
    dt = 0.4 * h[0] / v
    sigma = 20.0  # damping rate eta/m in 1/s
    m = np.full(shape, 1.0 / v ** 2, dtype=np.float32)
    eta = np.full(shape, np.float32(float(m.flat[0]) * sigma), dtype=np.float32)
    c = dt ** 2 / float(m.flat[0])
    d = dt * float(eta.flat[0]) / float(m.flat[0])
    p = (1, 2, 1)
    mode = dirichlet_mode(shape, p)
    lam = sum(4.0 / h[a] ** 2 * math.sin(math.pi * p[a] / (2 * (shape[a] + 1))) ** 2 for a in range(3))
    # amplitude recurrence a^{n+1} = (2 - d - c lam) a^n - (1 - d) a^{n-1}
    b = 2.0 - d - c * lam
    roots = np.roots([1.0, -b, 1.0 - d]).astype(complex)
    a0, am1 = 1.0, 0.6
    A = np.array([[1.0, 1.0], [1.0 / roots[0], 1.0 / roots[1]]])
    alpha = np.linalg.solve(A, np.array([a0, am1], dtype=complex))
    nsteps = 60
    u, up, _ = orc.acoustic_forward(shape, h, (0, 0, 0), 2, m, eta, dt, nsteps,
                                    u_cur=a0 * mode, u_prev=am1 * mode)
    an = (alpha * roots ** nsteps).sum().real
    np.testing.assert_allclose(u, an * mode, rtol=0, atol=1e-12)
    # the modulus of both roots is sqrt(1 - d): the envelope decays like
    # (1 - sigma dt)^{n/2} ~ exp(-sigma t / 2), the continuous damped oscillator
    assert np.allclose(np.abs(roots), math.sqrt(1.0 - d), rtol=1e-12)
    rate = math.log(math.sqrt(1.0 - d)) / dt
    assert abs(rate - (-sigma / 2)) < 0.5 * sigma * (sigma * dt)


def energy(orc, u_new, u_old, m, h, so, dt):
    du = u_new - u_old
    Lu = orc.laplacian(u_old, h, so)
    return float((m.astype(np.float64) * du * du).sum() / dt ** 2 - (u_new * Lu).sum())


@pytest.mark.parametrize("so", [4, 8])
def test_energy_conserved_without_damping(orc, so):
    shape = (18, 16, 20)
    h = (10.0, 10.0, 10.0)
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    m = (1.0 / v ** 2).astype(np.float32)
    dt = 0.4 * h[0] / 2500.0
    u0 = wl.random_field(shape, 1, smooth=2).astype(np.float64)
    u_cur, u_prev = u0.copy(), u0.copy()
    E = []
    for step in range(300):
        nc, npv, _ = orc.acoustic_forward(shape, h, (0, 0, 0), so, m, None, dt, 1,
                                          u_cur=u_cur, u_prev=u_prev, t0=step)
        E.append(energy(orc, nc, npv, m, h, so, dt))
        u_cur, u_prev = nc, npv
    E = np.array(E)
    assert (E > 0).all()
    assert np.abs(E / E[0] - 1).max() < 1e-12


def test_energy_decays_with_damping(orc):
    shape = (16, 16, 16)
    h = (10.0, 10.0, 10.0)
    v = np.full(shape, 2000.0)
    m = (1.0 / v ** 2).astype(np.float32)
    dt = 0.4 * h[0] / 2000.0
    # sponge scaled so that dt*eta/m stays near 0.1 per axis as in the 512^3 model
    sig = 0.12 * wl.sponge_sigma(shape, h, 5, 2000.0)
    eta = (m.astype(np.float64) * sig).astype(np.float32)
    u0 = wl.random_field(shape, 2, smooth=2).astype(np.float64)
    u_cur, u_prev = u0.copy(), u0.copy()
    E = []
    for step in range(120):
        nc, npv, _ = orc.acoustic_forward(shape, h, (0, 0, 0), 4, m, eta, dt, 1,
                                          u_cur=u_cur, u_prev=u_prev, t0=step)
        E.append(energy(orc, nc, npv, m, h, 4, dt))
        u_cur, u_prev = nc, npv
    E = np.array(E)
    assert (np.diff(E) <= 1e-12 * E[0]).all()
    assert E[-1] < 0.9 * E[0]


def test_injection_is_src_dt2_over_m(orc):
    """One step from rest: an on-node source adds src*dt^2/m at that node only;
    an off-node one spreads it with the linear weights, dt^2/m per corner."""
    shape = (9, 10, 11)
    h = (5.0, 4.0, 3.0)
    g = np.random.default_rng(5)
    m = (1.0 / g.uniform(1500, 3000, shape) ** 2).astype(np.float32)
    dt = 1e-3
    src = np.array([[0.75]])
    node = (4, 3, 7)
    u, _, rec = orc.acoustic_forward(shape, h, (0, 0, 0), 8, m, None, dt, 1,
                                     src_coords=np.array([[node[0] * h[0], node[1] * h[1], node[2] * h[2]]]),
                                     src_trace=src, rec_coords=np.array([[1.0, 1.0, 1.0]]))
    expect = np.zeros(shape)
    expect[node] = 0.75 * dt ** 2 / float(m[node])
    np.testing.assert_allclose(u, expect, rtol=1e-15, atol=0)
    assert rec[0, 0] == 0.0  # recorded from u^0 = 0
    # off node: fractions (0.25, 0.5, 0.1)
    x = np.array([[(2 + 0.25) * h[0], (5 + 0.5) * h[1], (3 + 0.1) * h[2]]])
    u, _, _ = orc.acoustic_forward(shape, h, (0, 0, 0), 8, m, None, dt, 1, src_coords=x, src_trace=src)
    for b0 in (0, 1):
        for b1 in (0, 1):
            for b2 in (0, 1):
                w = (0.25 if b0 else 0.75) * (0.5 if b1 else 0.5) * (0.1 if b2 else 0.9)
                at = (2 + b0, 5 + b1, 3 + b2)
                np.testing.assert_allclose(u[at], 0.75 * w * dt ** 2 / float(m[at]), rtol=1e-12)
    assert np.count_nonzero(u) == 8


def _adjoint_case(ndim, so, n, nt, seed):
    shape = (n + 2, n, n + 1)[:ndim]
    h = (10.0,) * ndim
    origin = (0.0,) * ndim
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    m = (1.0 / v ** 2).astype(np.float32)
    sig = wl.sponge_sigma(shape, h, 4, 2500.0, ref_width=40)
    eta = (m.astype(np.float64) * sig).astype(np.float32)
    dt = 0.4 * 10.0 / 2500.0
    src_c = wl.random_points(shape, h, origin, 3, seed)
    rec_c = wl.random_points(shape, h, origin, 5, seed + 1)
    g = np.random.default_rng(seed)
    s = g.standard_normal((nt, 3))
    r = g.standard_normal((nt, 5))
    return shape, h, origin, m, eta, dt, src_c, rec_c, s, r


@pytest.mark.parametrize("ndim,so", [(2, 4), (2, 16), (3, 8), (3, 2)])
def test_adjoint_dot_product(orc, ndim, so):
    shape, h, origin, m, eta, dt, src_c, rec_c, s, r = _adjoint_case(ndim, so, 14, 40, 3 + so)
    _, _, rec = orc.acoustic_forward(shape, h, origin, so, m, eta, dt, 40,
                                     src_coords=src_c, src_trace=s, rec_coords=rec_c)
    srca, _ = orc.acoustic_adjoint(shape, h, origin, so, m, eta, dt, 40, rec_c, r, src_c)
    lhs = float((rec * r).sum())
    rhs = float((s * srca).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs)), (lhs, rhs)
    assert abs(lhs) > 0


def test_adjoint_dot_product_fp32(orc):
    shape, h, origin, m, eta, dt, src_c, rec_c, s, r = _adjoint_case(3, 8, 14, 40, 7)
    s32, r32 = s.astype(np.float32), r.astype(np.float32)
    _, _, rec = orc.acoustic_forward(shape, h, origin, 8, m, eta, dt, 40, src_coords=src_c,
                                     src_trace=s32, rec_coords=rec_c, precision="f32")
    srca, _ = orc.acoustic_adjoint(shape, h, origin, 8, m, eta, dt, 40, rec_c, r32, src_c,
                                   precision="f32")
    lhs = float((rec.astype(np.float64) * r32).sum())
    rhs = float((s32.astype(np.float64) * srca).sum())
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))


def test_adjoint_is_explicit_transpose(orc):
    shape, h, origin, m, eta, dt, src_c, rec_c, _, _ = _adjoint_case(3, 4, 5, 6, 21)
    src_c, rec_c = src_c[:2], rec_c[:3]
    nt = 6
    F = np.zeros((nt * 3, nt * 2))
    for j in range(nt * 2):
        s = np.zeros(nt * 2)
        s[j] = 1.0
        _, _, rec = orc.acoustic_forward(shape, h, origin, 4, m, eta, dt, nt, src_coords=src_c,
                                         src_trace=s.reshape(nt, 2), rec_coords=rec_c)
        F[:, j] = rec.ravel()
    A = np.zeros((nt * 2, nt * 3))
    for j in range(nt * 3):
        r = np.zeros(nt * 3)
        r[j] = 1.0
        srca, _ = orc.acoustic_adjoint(shape, h, origin, 4, m, eta, dt, nt, rec_c, r.reshape(nt, 3), src_c)
        A[:, j] = srca.ravel()
    assert np.abs(F).max() > 0
    np.testing.assert_allclose(A, F.T, rtol=0, atol=1e-13 * np.abs(F).max())


def test_resume_is_bitwise(orc):
    cfg = wl.acoustic_config(n=20, space_order=4, nt=30, sponge=4, nrec_side=5)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 4, cfg["m"], cfg["eta"], cfg["dt"])
    u1, p1, r1 = orc.acoustic_forward(*args, 30, src_coords=cfg["src_coords"], src_trace=cfg["src_trace"],
                                      rec_coords=cfg["rec_coords"])
    ua, pa, ra = orc.acoustic_forward(*args, 12, src_coords=cfg["src_coords"], src_trace=cfg["src_trace"],
                                      rec_coords=cfg["rec_coords"], n_total=30)
    ub, pb, rb = orc.acoustic_forward(*args, 18, src_coords=cfg["src_coords"], src_trace=cfg["src_trace"],
                                      rec_coords=cfg["rec_coords"], u_cur=ua, u_prev=pa, t0=12, n_total=30)
    np.testing.assert_array_equal(u1, ub)
    np.testing.assert_array_equal(p1, pb)
    np.testing.assert_array_equal(r1[:12], ra[:12])
    np.testing.assert_array_equal(r1[12:], rb[12:])


def test_fp32_agrees_with_fp64(orc):
    cfg = wl.acoustic_config(n=24, space_order=8, nt=60, sponge=5, nrec_side=6)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["dt"], 60)
    kw = dict(src_coords=cfg["src_coords"], src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"])
    u64, _, r64 = orc.acoustic_forward(*args, **kw)
    u32, _, r32 = orc.acoustic_forward(*args, precision="f32", **kw)
    rel = np.linalg.norm(u32 - u64) / np.linalg.norm(u64)
    relr = np.linalg.norm(r32 - r64) / np.linalg.norm(r64)
    assert rel < 1e-5 and relr < 1e-5, (rel, relr)


def test_step_points_matches_loop_nest(orc):
    """The sampled single-step routine equals the full loop nest's step."""
    cfg = wl.acoustic_config(n=16, space_order=8, nt=1, sponge=3, nrec_side=3)
    shape = cfg["shape"]
    u = wl.random_field(shape, 4)
    up = wl.random_field(shape, 5)
    full, _, _ = orc.acoustic_forward(shape, cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"],
                                      cfg["dt"], 1, u_cur=u.astype(np.float64), u_prev=up.astype(np.float64))
    idx = np.arange(0, u.size, 7)
    pts = orc.step_points(shape, cfg["spacing"], 8, cfg["m"], cfg["eta"], cfg["dt"], u, up, idx)
    np.testing.assert_allclose(pts, full.ravel()[idx], rtol=1e-13, atol=1e-13 * np.abs(full).max())
