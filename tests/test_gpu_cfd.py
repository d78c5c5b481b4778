"""The Linear Convection and Laplace operators, and temporal blocking of the
small-grid cluster kernels, on the GPU against the oracle.

Fields are FP32 on both sides (the oracle's FP32 loop nest, no FMA); the GPU
contracts to FMA, so single steps agree to a few ulp and runs to 1e-5 of the
field's maximum.  The cluster kernels compute the same per-point arithmetic
for every number of steps between exchanges, and in the same order as the
plain per-step kernels, so those results agree bit for bit.  The convergence loop sums |p| in FP64 on both sides and stops at the
same sweep unless the two r straddle tol within their FP32 difference.
"""
import numpy as np
import pytest

import oracle
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class Run2D:
    def __init__(self, kind, so, u0, spacing, a=0.0, flags=0):
        torch = _torch()
        from paper_1707_03776_gb300 import fd
        self.fd = fd
        self.grid = fd.Grid(u0.shape, spacing)
        self.u = fd.TimeData("u", self.grid)
        self.u.at(0).copy_(torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)))
        self.op = fd.Operator(kind, so, self.u, a=a, flags=flags)

    def run(self, t0, nt, dt):
        self.op.apply(t0, nt, dt)
        self.op.sync()
        return self.u.at(t0 + nt).cpu().numpy().copy(), self.u.at(t0 + nt - 1).cpu().numpy().copy()


def _conv_case(shape, seed):
    g = np.random.default_rng(seed)
    u0 = g.standard_normal(shape).astype(np.float32)
    return u0, (0.1, 0.12), 1.0, 0.04  # nu = 0.4 + 0.333


@pytest.mark.parametrize("shape", [(41, 37), (254, 254), (300, 700), (7, 5)])
def test_convection_parity_and_time_blocks(shape):
    from paper_1707_03776_gb300 import fd
    u0, h, c, dt = _conv_case(shape, 1)
    ref = oracle.convection(u0, h, c, dt, 23, precision="f32")
    ref_prev = oracle.convection(u0, h, c, dt, 22, precision="f32")
    scale = np.abs(ref).max()
    outs = []
    for k in (0, 1, 2, 5):
        run = Run2D(fd.FD_CONVECTION_UPWIND, 1, u0, h, a=c)
        if k:
            try:
                fd.fd_operator_set_time_block(run.op.handle, k)
            except fd.FDError as e:
                assert e.status == fd.FD_ERR_UNSUPPORTED
                continue
        last, prev = run.run(0, 23, dt)
        assert np.abs(last - ref).max() <= 1e-5 * scale
        assert np.abs(prev - ref_prev).max() <= 1e-5 * scale
        outs.append(last)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    plain = Run2D(fd.FD_CONVECTION_UPWIND, 1, u0, h, a=c, flags=fd.FD_FLAG_PLAIN_KERNELS)
    last, _ = plain.run(0, 23, dt)
    assert np.abs(last - ref).max() <= 1e-5 * scale


@pytest.mark.parametrize("kind,so", [("diffusion", 2), ("diffusion", 4), ("convection", 1)])
def test_cluster_and_plain_kernels_agree_bitwise(kind, so):
    """One cluster launch for the whole run (K steps per exchange; at SO2 4
    columns per thread on the paired FP32 instructions) and one launch of the
    plain kernel per step do the same arithmetic per point in the same order,
    so the fields agree bit for bit after many steps."""
    from paper_1707_03776_gb300 import fd
    if kind == "diffusion":
        cfg = wl.diffusion_ring(courant=0.1)
        args, a, dt, nt = (fd.FD_DIFFUSION_EULER, so, cfg["u0"], cfg["spacing"]), cfg["a"], cfg["dt"], 61
    else:
        u0, h, c, dt = _conv_case((83, 77), 3)
        args, a, nt = (fd.FD_CONVECTION_UPWIND, 1, u0, h), c, 29
    fast = Run2D(*args, a=a)
    plain = Run2D(*args, a=a, flags=fd.FD_FLAG_PLAIN_KERNELS)
    f_last, f_prev = fast.run(0, nt, dt)
    p_last, p_prev = plain.run(0, nt, dt)
    assert np.abs(f_last).max() > 0
    np.testing.assert_array_equal(f_last, p_last)
    np.testing.assert_array_equal(f_prev, p_prev)


def test_convection_example_workload():
    """The paper's example (81^2, c = 1, 100 steps) against the FP64 oracle."""
    from paper_1707_03776_gb300 import fd
    cfg = wl.convection_config()
    run = Run2D(fd.FD_CONVECTION_UPWIND, 1, cfg["u0"], cfg["spacing"], a=cfg["c"])
    k, ctas = fd.fd_operator_get_time_block(run.op.handle)
    assert k >= 1 and ctas >= 1
    last, _ = run.run(0, cfg["nt"], cfg["dt"])
    ref = oracle.convection(cfg["u0"].astype(np.float64), cfg["spacing"], cfg["c"], cfg["dt"], cfg["nt"])
    assert np.linalg.norm(last - ref) <= 1e-5 * np.linalg.norm(ref)
    # the bump moved by c t = 0.5 along x and y and lost height to numerical diffusion
    i, j = np.unravel_index(np.argmax(last), last.shape)
    h = cfg["spacing"][0]
    assert abs(i * h - 1.25) <= 2 * h and abs(j * h - 1.25) <= 2 * h
    assert 0.5 < last.max() < 1.0


def test_convection_errors():
    from paper_1707_03776_gb300 import fd
    u0, h, c, dt = _conv_case((20, 20), 2)
    run = Run2D(fd.FD_CONVECTION_UPWIND, 1, u0, h, a=c)
    with pytest.raises(fd.FDError) as e:
        run.op.apply(0, 1, 0.1)  # c dt (1/dx + 1/dy) > 1
    assert e.value.status == fd.FD_ERR_UNSTABLE
    with pytest.raises(fd.FDError) as e:
        Run2D(fd.FD_CONVECTION_UPWIND, 2, u0, h, a=c)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [(25, 13), (31, 31), (200, 180), (600, 90)])
def test_laplace_sweeps_parity(shape):
    from paper_1707_03776_gb300 import fd
    g = np.random.default_rng(3)
    p0 = g.standard_normal(shape).astype(np.float32)
    sp = (2.0 / (shape[0] - 1), 1.0 / (shape[1] - 1))
    ref, _, _ = oracle.laplace(p0, sp, 0.0, 17, precision="f32")
    scale = np.abs(ref).max()
    outs = []
    for flags, k in ((0, 0), (0, 1), (0, 3), (fd.FD_FLAG_PLAIN_KERNELS, 0)):
        run = Run2D(fd.FD_LAPLACE_JACOBI, 2, p0, sp, flags=flags)
        if k:
            try:
                fd.fd_operator_set_time_block(run.op.handle, k)
            except fd.FDError:
                continue
        last, _ = run.run(0, 17, 0.0)
        assert np.abs(last - ref).max() <= 1e-5 * scale
        if not flags:
            outs.append(last)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("flags", [0, "plain"])
@pytest.mark.parametrize("shape", [(31, 31), (120, 70)])
def test_laplace_convergence_loop(flags, shape):
    from paper_1707_03776_gb300 import fd
    cfg = wl.laplace_config(nx=shape[0], ny=shape[1])
    fl = fd.FD_FLAG_PLAIN_KERNELS if flags == "plain" else 0
    run = Run2D(fd.FD_LAPLACE_JACOBI, 2, cfg["p0"], cfg["spacing"], flags=fl)
    it, r = run.op.converge(0, 200000, cfg["tol"])
    got = run.u.at(it).cpu().numpy()
    ref, it_ref, r_ref = oracle.laplace(cfg["p0"], cfg["spacing"], cfg["tol"], 200000, precision="f32")
    assert r < cfg["tol"] and it < 200000
    if it != it_ref:
        # only when the two r straddle tol within their FP32 difference
        assert abs(it - it_ref) == 1 and abs(r_ref - cfg["tol"]) <= 1e-6 * cfg["tol"] + abs(r - r_ref)
    else:
        assert abs(r - r_ref) <= 1e-3 * r_ref
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    # the steady state approaches the linear profile in y at x = 2 and 0 at x = 0
    assert np.all(got[0] == 0.0)


@pytest.mark.parametrize("shape", [(31, 31), (120, 70)])
def test_laplace_stops_at_max_iter(shape):
    """A loop cut off by max_iter before the criterion: the sweeps done, the
    field and the last r (formed from the final two sums) against the oracle;
    then zero sweeps leave everything as it was."""
    from paper_1707_03776_gb300 import fd
    cfg = wl.laplace_config(nx=shape[0], ny=shape[1])
    run = Run2D(fd.FD_LAPLACE_JACOBI, 2, cfg["p0"], cfg["spacing"])
    it, r = run.op.converge(0, 37, cfg["tol"])
    ref, it_ref, r_ref = oracle.laplace(cfg["p0"], cfg["spacing"], cfg["tol"], 37, precision="f32")
    assert it == it_ref == 37 and r > cfg["tol"]
    assert abs(r - r_ref) <= 1e-4 * r_ref
    got = run.u.at(it).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()
    it0, r0 = run.op.converge(37, 0, cfg["tol"])
    assert it0 == 0
    np.testing.assert_array_equal(run.u.at(37).cpu().numpy(), got)


def test_diffusion_time_blocks_agree_bitwise():
    from paper_1707_03776_gb300 import fd
    cfg = wl.diffusion_ring()
    ref = oracle.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], 57, precision="f32")
    outs = []
    for k in (0, 1, 2, 4):
        run = Run2D(fd.FD_DIFFUSION_EULER, 2, cfg["u0"], cfg["spacing"], a=cfg["a"])
        if k:
            fd.fd_operator_set_time_block(run.op.handle, k)
            assert fd.fd_operator_get_time_block(run.op.handle)[0] == k
        last, _ = run.run(0, 57, cfg["dt"])
        assert np.abs(last - ref).max() <= 1e-5
        outs.append(last)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    with pytest.raises(fd.FDError) as e:
        fd.fd_operator_set_time_block(run.op.handle, 200)
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
