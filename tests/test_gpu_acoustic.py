"""Parity of the CUDA acoustic path (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 <= 1e-6 for the field after one step, <= 1e-4 for
receiver traces after a full run (FP32 kernels against FP64 loop nests on the
same FP32 inputs).  Shapes span several tiles (64 columns, up to 32 rows) and
ragged tails in every axis; both the tiled TMA kernel and the plain kernel are
checked.
"""
import numpy as np
import pytest

import oracle
from fdrun import AcousticRun, rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ONE_STEP_TOL = 1e-6
TRACE_TOL = 1e-4


def _model(shape, h, sponge, seed):
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    m = (1.0 / v ** 2).astype(np.float32)
    sig = wl.sponge_sigma(shape, (h,) * len(shape), sponge, 2500.0, ref_width=40)
    eta = (m.astype(np.float64) * sig).astype(np.float32)
    return m, eta, 0.4 * h / 2500.0


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS], ids=["tiled", "plain"])
@pytest.mark.parametrize("so,shape", [
    (2, (9, 40, 70)), (4, (21, 70, 150)), (8, (33, 67, 131)), (16, (20, 45, 200)),
    (8, (5, 6, 7)), (8, (2, 33, 64)), (12, (17, 96, 128)),
    (4, (67, 133)), (16, (40, 90)),
])
def test_one_step_parity(so, shape, flags):
    h = 10.0
    m, eta, dt = _model(shape, h, 4, 1)
    u = wl.random_field(shape, 10 + so, smooth=1)
    up = wl.random_field(shape, 20 + so, smooth=1)
    run = AcousticRun(shape, (h,) * len(shape), None, so, m, eta, flags=flags)
    run.set_state(u, up)
    run.run(0, 1, dt)
    got, _ = run.state(1)
    ref, _, _ = oracle.acoustic_forward(shape, (h,) * len(shape), (0,) * len(shape), so, m, eta, dt, 1,
                                        u_cur=u.astype(np.float64), u_prev=up.astype(np.float64))
    err = rel_l2(got, ref)
    assert err <= ONE_STEP_TOL, err


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS], ids=["tiled", "plain"])
@pytest.mark.parametrize("so", [4, 8, 16])
def test_full_run_traces(so, flags):
    """Source at the surface centre, a receiver lattice, sponge, many steps."""
    cfg = wl.acoustic_config(n=48, space_order=so, nt=220, sponge=8, nrec_side=9)
    run = AcousticRun(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["m"], cfg["eta"],
                      cfg["src_coords"], cfg["src_trace"], cfg["rec_coords"], cfg["nt"], flags=flags)
    run.run(0, cfg["nt"], cfg["dt"])
    rec = run.rec_trace()
    u_end, _ = run.state(cfg["nt"])
    ou, _, orec = oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["m"],
                                          cfg["eta"], cfg["dt"], cfg["nt"], src_coords=cfg["src_coords"],
                                          src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"])
    assert np.abs(orec).max() > 0
    assert rel_l2(rec, orec) <= TRACE_TOL
    assert rel_l2(u_end, ou) <= TRACE_TOL
    assert run.op.launches > cfg["nt"]


def test_two_dimensional_run():
    cfg = wl.acoustic_config(n=120, space_order=8, nt=200, sponge=10, nrec_side=31, ndim=2)
    run = AcousticRun(cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"],
                      cfg["src_coords"], cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    run.run(0, cfg["nt"], cfg["dt"])
    _, _, orec = oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"],
                                         cfg["dt"], cfg["nt"], src_coords=cfg["src_coords"],
                                         src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"])
    assert rel_l2(run.rec_trace(), orec) <= TRACE_TOL


def test_adjoint_matches_oracle_and_dot_product():
    """FD_FLAG_REVERSE with swapped point sets is the oracle's adjoint, and the
    GPU forward/adjoint pair passes the dot-product test."""
    import torch
    shape, h, so, nt = (30, 34, 40), 10.0, 8, 80
    m, eta, dt = _model(shape, h, 5, 3)
    g = np.random.default_rng(5)
    src_c = wl.random_points(shape, (h,) * 3, (0, 0, 0), 3, 31)
    rec_c = wl.random_points(shape, (h,) * 3, (0, 0, 0), 7, 32)
    s = g.standard_normal((nt, 3)).astype(np.float32)
    r = g.standard_normal((nt, 7)).astype(np.float32)
    fwd = AcousticRun(shape, (h,) * 3, None, so, m, eta, src_c, s, rec_c, nt)
    fwd.run(0, nt, dt)
    d_rec = fwd.rec_trace()
    # adjoint: inject r at receivers, record at sources, backward in time from rest
    adj = AcousticRun(shape, (h,) * 3, None, so, m, eta, rec_c, r, src_c, nt, flags=fd.FD_FLAG_REVERSE)
    adj.run(0, nt, dt)
    srca = adj.rec_trace()
    o_srca, _ = oracle.acoustic_adjoint(shape, (h,) * 3, (0, 0, 0), so, m, eta, dt, nt, rec_c, r, src_c)
    assert rel_l2(srca, o_srca) <= TRACE_TOL
    lhs = float((d_rec.astype(np.float64) * r).sum())
    rhs = float((s.astype(np.float64) * srca).sum())
    assert abs(lhs - rhs) <= 1e-4 * max(abs(lhs), abs(rhs))
    torch.cuda.synchronize()


def test_resume_is_bitwise():
    cfg = wl.acoustic_config(n=40, space_order=8, nt=30, sponge=6, nrec_side=5)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    a = AcousticRun(*args)
    a.run(0, 30, cfg["dt"])
    b = AcousticRun(*args)
    b.run(0, 12, cfg["dt"])
    b.run(12, 18, cfg["dt"])
    ua, pa = a.state(30)
    ub, pb = b.state(30)
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(a.rec_trace(), b.rec_trace())


def test_tiled_equals_plain_closely():
    cfg = wl.acoustic_config(n=64, space_order=8, nt=50, sponge=8, nrec_side=7)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    a = AcousticRun(*args)
    a.run(0, 50, cfg["dt"])
    b = AcousticRun(*args, flags=fd.FD_FLAG_PLAIN_KERNELS)
    b.run(0, 50, cfg["dt"])
    assert rel_l2(a.state(50)[0], b.state(50)[0]) < 1e-5


@pytest.mark.parametrize("so,shape", [(4, (21, 70, 150)), (8, (33, 67, 131)), (12, (17, 96, 128)),
                                      (16, (20, 45, 200))])
def test_tiled_equals_plain_bitwise_without_sources(so, shape):
    """Without sources (fused and atomic injection round differently) the
    tiled kernel -- TMA tiles, the register queue, the Laplacian on paired
    FP32 instructions -- and the plain kernel do the same arithmetic per point
    in the same order, so fields and receiver traces agree bit for bit."""
    h, nt = 10.0, 12
    m, eta, dt = _model(shape, h, 6, 0)
    rec = wl.random_points(shape, (h,) * 3, (0.0,) * 3, 37, 5)
    args = (shape, (h,) * 3, (0.0,) * 3, so, m, eta, None, None, rec, nt)
    u1 = wl.random_field(shape, 11, smooth=2)
    u0 = wl.random_field(shape, 12, smooth=2)
    a = AcousticRun(*args)
    b = AcousticRun(*args, flags=fd.FD_FLAG_PLAIN_KERNELS)
    for r in (a, b):
        r.set_state(u1, u0)
        r.run(0, nt, dt)
    ua, pa = a.state(nt)
    ub, pb = b.state(nt)
    assert np.abs(ua).max() > 0
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(a.rec_trace(), b.rec_trace())


def test_zero_steps_and_errors():
    shape, h = (16, 17, 18), 10.0
    m, eta, dt = _model(shape, h, 3, 4)
    run = AcousticRun(shape, (h,) * 3, None, 8, m, eta)
    u = wl.random_field(shape, 3)
    run.set_state(u, u)
    run.run(0, 0, dt)
    np.testing.assert_array_equal(run.state(0)[0], u)
    with pytest.raises(fd.FDError) as e:
        run.op.apply(0, 1, 1.05 * dt / 0.4 * 2.0)  # far above the CFL limit
    assert e.value.status == fd.FD_ERR_UNSTABLE
    with pytest.raises(fd.FDError) as e:
        run.op.apply(0, 1, -1.0)
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    grid = fd.Grid(shape, (h,) * 3)
    with pytest.raises(fd.FDError) as e:
        fd.PointData("bad", grid, np.array([[0.0, 0.0, 17 * h + 1.0]]), 4)
    assert e.value.status == fd.FD_ERR_OUT_OF_DOMAIN
    src = fd.PointData("s", grid, np.array([[10.0, 10.0, 10.0]]), 4)
    u2 = fd.TimeData("u", grid)
    m2 = fd.DenseData("m", grid)
    m2.data.fill_(1.0 / 2000.0 ** 2)
    op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u2, m2, src=src)
    with pytest.raises(fd.FDError) as e:
        op.apply(2, 3, dt)  # needs 5 trace rows, has 4
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    with pytest.raises(fd.FDError) as e:
        fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 7, u2, m2)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
    other = fd.Grid((16, 17, 19), (h,) * 3)
    with pytest.raises(fd.FDError):
        fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u2, fd.DenseData("m", other))


def test_rebind_by_name():
    """op(m=...) style rebinding recomputes the coefficients."""
    shape, h = (20, 24, 28), 10.0
    m, eta, dt = _model(shape, h, 3, 6)
    run = AcousticRun(shape, (h,) * 3, None, 4, m, eta)
    u = wl.random_field(shape, 8, smooth=1)
    m2 = (m * np.float32(1.3)).astype(np.float32)
    newm = fd.DenseData("m", run.grid)
    import torch
    newm.data.copy_(torch.from_numpy(m2))
    run.op.bind("m", newm)
    run.set_state(u, u)
    run.run(0, 1, dt)
    ref, _, _ = oracle.acoustic_forward(shape, (h,) * 3, (0, 0, 0), 4, m2, eta, dt, 1,
                                        u_cur=u.astype(np.float64), u_prev=u.astype(np.float64))
    assert rel_l2(run.state(1)[0], ref) <= ONE_STEP_TOL


def test_rebind_u_keeps_the_fused_sources():
    """Rebinding u rebuilds the tiled plan and its fused source table with
    it: the run on the new field equals a fresh operator's bit for bit."""
    cfg = wl.acoustic_config(n=48, space_order=8, nt=12, sponge=4, nrec_side=3)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    run = AcousticRun(*args)
    u2 = fd.TimeData("u", run.grid)
    run.op.bind("u", u2)
    run.u = u2
    run.run(0, cfg["nt"], cfg["dt"])
    ref = AcousticRun(*args)
    ref.run(0, cfg["nt"], cfg["dt"])
    np.testing.assert_array_equal(run.state(cfg["nt"])[0], ref.state(cfg["nt"])[0])
    np.testing.assert_array_equal(run.rec_trace(), ref.rec_trace())
    assert np.abs(ref.rec_trace()).max() > 0


def test_tilings_agree_bitwise_and_autotune():
    """Every tiling (tile height, prefetch depth, d0 chunks) computes the same
    per-point arithmetic, so results agree bit for bit; the autotuner picks
    one of them."""
    cfg = wl.acoustic_config(n=72, space_order=8, nt=30, sponge=8, nrec_side=7)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    results = []
    for rows, stages in [(0, 0), (8, 2), (13, 3), (30, 4), (20, 2)]:
        run = AcousticRun(*args)
        fd.fd_operator_set_tiling(run.op.handle, rows, stages)
        r, s, ctas = fd.fd_operator_get_tiling(run.op.handle)
        assert r > 0 and s >= 2 and ctas > 0
        if rows:
            assert r <= rows and s == stages
            # 72 planes of 2 x ceil(72/r) columns do not fill the GPU: the
            # planner splits d0 into chunks swept by separate CTAs
            assert ctas >= 2 * (2 * -(-72 // r))
        run.run(0, 30, cfg["dt"])
        results.append((run.state(30)[0], run.rec_trace()))
    for u, rec in results[1:]:
        np.testing.assert_array_equal(u, results[0][0])
        np.testing.assert_array_equal(rec, results[0][1])
    run = AcousticRun(*args)
    rows, stages, ms = fd.fd_operator_autotune(run.op.handle, 0, 5, cfg["dt"])
    assert rows in (8, 10, 12, 14, 16, 18, 20, 24, 27, 30) and 2 <= stages <= 4 and ms > 0
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_set_tiling(run.op.handle, 64, 2)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
    assert fd.fd_operator_get_tiling(run.op.handle)[:2] == (rows, stages)


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS], ids=["tiled", "plain"])
@pytest.mark.parametrize("so,shape", [
    (2, (2, 2, 2)), (16, (3, 5, 2)), (8, (2, 2, 9)), (4, (2, 70, 3)), (16, (17, 2, 65)),
    (2, (2, 2)), (16, (2, 40)), (8, (3, 3)),
])
def test_degenerate_shapes(so, shape, flags):
    """The smallest grids (2 nodes per axis), grids thinner than the
    stencil's half-width and contiguous axes of 2-3 points (TMA boxes almost
    entirely outside the grid): the zero halo still gives the oracle's
    result.  A source on the grid's last node and a receiver on its first
    exercise the interpolation table's clamp."""
    h = 10.0
    nd = len(shape)
    m, eta, dt = _model(shape, h, 0, 2)
    u = wl.random_field(shape, 30 + so, smooth=0)
    up = wl.random_field(shape, 40 + so, smooth=0)
    hi = np.array([(n - 1) * h for n in shape], dtype=np.float64).reshape(1, nd)
    lo = np.zeros((1, nd))
    nt = 3
    src_trace = np.linspace(1.0, 2.0, nt).astype(np.float32).reshape(nt, 1)
    run = AcousticRun(shape, (h,) * nd, None, so, m, eta, src_coords=hi, src_trace=src_trace, rec_coords=lo,
                      n_total=nt, flags=flags | fd.FD_FLAG_NO_CFL_CHECK)
    run.set_state(u, up)
    run.run(0, nt, dt)
    got, _ = run.state(nt)
    ref, _, rec = oracle.acoustic_forward(shape, (h,) * nd, (0,) * nd, so, m, eta, dt, nt, src_coords=hi,
                                          src_trace=src_trace, rec_coords=lo, u_cur=u.astype(np.float64),
                                          u_prev=up.astype(np.float64))
    assert rel_l2(got, ref) <= 1e-5
    np.testing.assert_allclose(run.rec_trace()[:, 0], rec[:, 0], rtol=1e-5, atol=1e-6 * np.abs(rec).max())


@pytest.mark.parametrize("so", [4, 8, 16])
def test_full_run_128(so):
    """The 512^3 benchmark's recipe at 128^3 x 300 steps (40-cell-strength
    sponge of 16 cells, 33 x 33 receivers): receiver traces and the final
    field against the FP64 oracle's full run, relative L2 <= 1e-4; the
    planner's tiling (d0 chunks at this size) as the bench uses it."""
    cfg = wl.acoustic_config(n=128, space_order=so, nt=300, sponge=16, nrec_side=33)
    run = AcousticRun(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["m"], cfg["eta"],
                      cfg["src_coords"], cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    rows, stages, ctas = fd.fd_operator_get_tiling(run.op.handle)
    assert ctas >= 152  # the columns alone would leave SMs idle: d0 chunks
    run.run(0, cfg["nt"], cfg["dt"])
    rec = run.rec_trace()
    u_end, _ = run.state(cfg["nt"])
    ou, _, orec = oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["m"],
                                          cfg["eta"], cfg["dt"], cfg["nt"], src_coords=cfg["src_coords"],
                                          src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"])
    assert np.abs(orec).max() > 0
    assert rel_l2(rec, orec) <= TRACE_TOL
    assert rel_l2(u_end, ou) <= TRACE_TOL


def test_bounded_wait_gives_up_and_reports():
    """The failure path on the GPU without a fault: the stall hook arms one
    tile's barrier for a u^n plane whose copy is never issued, so that CTA's
    bounded wait (2 s) runs out; it records FD_ERR_TIMEOUT, drains the copies
    it did issue (one shared 2 s deadline) and returns, the host reads the status at sync, and the next run (hook
    off) is correct again."""
    import time
    cfg = wl.acoustic_config(n=40, space_order=8, nt=6, sponge=4, nrec_side=3)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    run = AcousticRun(*args)
    fd.fd_operator_debug_stall(run.op.handle, 5)
    t0 = time.perf_counter()
    # the first launch waits 2 s, then drains for 2 s; the second sees the
    # status word set and returns at once
    run.op.apply(0, 2, cfg["dt"])
    with pytest.raises(fd.FDError) as e:
        run.op.sync()
    assert e.value.status == fd.FD_ERR_TIMEOUT
    assert 3.5 < time.perf_counter() - t0 < 30.0
    # the status was cleared by the sync: with the hook off the run is exact
    fd.fd_operator_debug_stall(run.op.handle, -1)
    for s in run.u.slots:
        s.zero_()
    run.run(0, cfg["nt"], cfg["dt"])
    ref = AcousticRun(*args)
    ref.run(0, cfg["nt"], cfg["dt"])
    np.testing.assert_array_equal(run.state(cfg["nt"])[0], ref.state(cfg["nt"])[0])
    np.testing.assert_array_equal(run.rec_trace(), ref.rec_trace())


def test_forward_with_receivers_beside_is_reproducible():
    """Runs of 16 steps or more interpolate the receivers on a side stream,
    concurrently with the grid update; the results must not depend on how
    the two kernels share the SMs.  Three runs of a 256^3 forward (65 x 65
    receivers, d0 chunks) give the same fields and traces bit for bit.  (A
    refill of the tiled kernel's ring slots not fenced against the compute
    warps' reads made them differ.)"""
    from paper_1707_03776_gb300.modeling import AcousticModel
    cfg = wl.gradient_config(n=256, nt=120)
    out = []
    for _ in range(3):
        model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["shots"][0], cfg["rec_coords"],
                              cfg["nt"])
        model.load(cfg["m_true"], cfg["eta"], cfg["wavelet"])
        model.run(cfg["dt"])
        model.op.sync()
        out.append((model.rec.data[:, : model.rec.npoint].cpu().numpy(), model.u.at(cfg["nt"]).cpu().numpy()))
        del model
    for rec, u in out[1:]:
        np.testing.assert_array_equal(rec, out[0][0])
        np.testing.assert_array_equal(u, out[0][1])
    assert np.abs(out[0][0]).max() > 0
