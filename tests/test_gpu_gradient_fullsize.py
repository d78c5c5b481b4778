"""The gradient workload at its configured size: 256^3 SO8, 1500 steps, 65 x 65
receivers, the starting model of the two-layer-plus-anomaly configuration,
checkpoints every 50 steps -- the run the gradient benchmark times, on the
first of its eight shots.  The configuration names the two checks below.
Both are properties of the exact operators that hold at any size, so no CPU
run of the oracle is needed at this size (the oracle pins the same
operators on small grids: test_gpu_gradient.py, test_oracle_gradient.py).

* The dot-product test of the Seismic Inversion Example: F maps the source
  wavelet s to the receiver traces at the starting model, F^T (the adjoint
  operator, FD_FLAG_REVERSE with the point sets swapped) maps receiver traces
  back to the source position, and <F s, r> = <s, F^T r>.  With r = F s the
  left side is |F s|^2, so neither side is a small difference of large terms.

* The objective J(m) = 1/2 |F(m) s - d_obs|^2, d_obs the traces of the true
  model, against its adjoint-state gradient g along dm = m_true - m0:
  - the Taylor remainder J(m0 + h dm) - J(m0) - h <g, dm> falls as h^2;
  - central differences c(h) = (J(m0 + h dm) - J(m0 - h dm)) / 2h at
    h = 0.4, 0.2, 0.1 (error A h^2 + B h^4 + ...), Richardson-extrapolated
    twice, equal <g, dm>.  J is far from quadratic along dm on this
    geometry (c(h) changes sign between h = 0.1 and 0.4), so a single
    extrapolation would leave an h^4 error of a few 1e-3.

Tolerances, from the FP32 arithmetic.  Receiver traces after a full run
carry a relative L2 error delta <= 1e-4 (the full-run gate of the 512^3
workload measured 3e-5 after 1000 steps).
  - Dot product: |F s|^2 then has relative error <= 2 delta.  <s, F^T F s> adds
    the adjoint run's delta on F^T r, amplified by
    kappa = sum |s_i (F^T r)_i| / |sum s_i (F^T r)_i|, the cancellation of
    that sum.  Bound: 2 delta (1 + kappa), with kappa measured.
  - Objective: the rounding error of J is measured, not bounded: the same
    objective through the plain kernels (another FP32 rounding of every
    step) differs from the tiled one by about that error.  The bound
    2 delta |d| |r| would be far too pessimistic, because the traces'
    rounding errors are not aligned with the residual r.  The Taylor ratios
    are checked where the remainder exceeds 20 times the measured error.
    The doubly extrapolated difference weighs the J values by at most
    (64/0.1 + 20/0.2 + 1/0.4) / 45 < 17 per unit of J error.  Twice the
    measured error times that enters its tolerance.
  - Gradient: <g, dm> sums mu^n (u^n - 2u^{n-1} + u^{n-2}) over 1500 steps.
    The second time difference divides the fields' relative error by
    (omega dt)^2, about 0.05 at the wavelet's upper frequency: 2e-3 per
    term, averaging down over the sum.  The gradient is therefore held to
    2e-3 of the extrapolated differences, plus their rounding.
"""
import numpy as np
import pytest

from fdrun import AcousticRun
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DELTA = 1e-4       # relative L2 error of receiver traces after a full run (FP32)
GRAD_TOL = 2e-3    # <g, dm> against the extrapolated central differences


@pytest.fixture(scope="module")
def cfg():
    return wl.gradient_config()


def test_forward_adjoint_dot_product_full_size(cfg):
    nt, dt = cfg["nt"], cfg["dt"]
    h = cfg["spacing"]
    src_c = cfg["shots"][0]
    rec_c = cfg["rec_coords"]
    s = cfg["wavelet"].astype(np.float32)
    fwd = AcousticRun(cfg["shape"], h, None, 8, cfg["m0"], cfg["eta"], src_c, s, rec_c, nt)
    fwd.run(0, nt, dt)
    r = fwd.rec_trace()
    del fwd
    # adjoint: r injected at the receivers, recorded at the source, backward in time from rest
    adj = AcousticRun(cfg["shape"], h, None, 8, cfg["m0"], cfg["eta"], rec_c, r, src_c, nt,
                      flags=fd.FD_FLAG_REVERSE)
    adj.run(0, nt, dt)
    sa = adj.rec_trace().astype(np.float64)
    del adj
    r64 = r.astype(np.float64)
    lhs = float((r64 * r64).sum())
    terms = s.astype(np.float64) * sa
    rhs = float(terms.sum())
    kappa = float(np.abs(terms).sum()) / abs(rhs)
    assert lhs > 0 and np.isfinite(kappa)
    tol = 2 * DELTA * (1 + kappa)
    print("dot product: relative mismatch %.3e, kappa %.2f, tolerance %.3e" % (abs(lhs - rhs) / lhs, kappa, tol))
    assert abs(lhs - rhs) <= tol * lhs, (lhs, rhs, kappa, abs(lhs - rhs) / lhs)


def test_gradient_taylor_and_central_differences_full_size(cfg):
    import torch
    from paper_1707_03776_gb300.gradient import Propagator, Shot, modelling
    nt, dt = cfg["nt"], cfg["dt"]
    prop = Propagator(cfg["shape"], cfg["spacing"], cfg["origin"], 8, Shot(cfg["shots"][0], cfg["wavelet"],
                      cfg["rec_coords"]), nt, dt, checkpoint_every=50)
    prop.set_damping(cfg["eta"])
    m_true = torch.from_numpy(cfg["m_true"]).cuda()
    m0 = torch.from_numpy(cfg["m0"]).cuda()
    prop.set_model(m_true)
    d_obs = prop.forward().clone()
    d64 = d_obs.double()

    def objective(m):
        prop.set_model(m)
        res = prop.forward().double() - d64
        return 0.5 * float((res * res).sum()), float(res.norm())

    m = m0.clone().requires_grad_(True)
    rec = modelling(m, prop)
    (0.5 * ((rec - d_obs) ** 2).sum()).backward()
    dm = m_true - m0
    gdm = float((m.grad.double() * dm.double()).sum())
    J0, rn = objective(m0)
    assert J0 > 0 and gdm != 0
    # the rounding error of J: the same objective through the plain kernels
    plain = Propagator(cfg["shape"], cfg["spacing"], cfg["origin"], 8, Shot(cfg["shots"][0], cfg["wavelet"],
                       cfg["rec_coords"]), nt, dt, checkpoint_every=50, flags=fd.FD_FLAG_PLAIN_KERNELS)
    plain.set_damping(cfg["eta"])
    plain.set_model(m0)
    res = plain.forward().double() - d64
    noise = abs(0.5 * float((res * res).sum()) - J0)
    del plain, res
    torch.cuda.empty_cache()

    hs = (0.4, 0.2, 0.1)
    Jp = [objective(m0 + hh * dm)[0] for hh in hs]
    Jm = [objective(m0 - hh * dm)[0] for hh in hs]
    # Taylor remainder: second order in h wherever it stands above the noise
    e2 = [abs(jp - J0 - hh * gdm) for jp, hh in zip(Jp, hs)]
    checked = 0
    for i in range(len(hs) - 1):
        if e2[i + 1] > 20 * noise:
            assert 2.8 <= e2[i] / e2[i + 1] <= 6.0, (e2, noise)
            checked += 1
    assert checked == len(hs) - 1, (e2, noise)
    # central differences, Richardson-extrapolated twice (h = 0.4, 0.2, 0.1)
    c = [(jp - jm) / (2 * hh) for jp, jm, hh in zip(Jp, Jm, hs)]
    r1 = [(4 * c[i + 1] - c[i]) / 3 for i in range(2)]
    c_star = (16 * r1[1] - r1[0]) / 15
    tol = GRAD_TOL + 2 * 17 * noise / abs(gdm)
    print("|r|/|d| %.3f; Taylor remainders %s (J rounding %.3e); central differences %s -> %.6e vs <g, dm> %.6e: "
          "relative %.3e, tolerance %.3e" % (rn / float(d64.norm()), ["%.4e" % e for e in e2], noise,
                                             ["%.6e" % x for x in c], c_star, gdm, abs(c_star - gdm) / abs(gdm), tol))
    assert abs(c_star - gdm) <= tol * abs(gdm), (c, c_star, gdm, abs(c_star - gdm) / abs(gdm))
