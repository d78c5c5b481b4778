"""Adjoint-state gradient on the GPU (checkpointed forward, recomputed
segments, reverse-time adjoint and imaging condition through the C ABI,
behind torch.autograd) against the FP64 oracle gradient, which is itself
pinned by central finite differences.

Tolerance: relative L2 <= 1e-3 on dJ/dm (FP32 wavefields summed over all
steps; each term carries ~1e-6 relative error from the forward and adjoint
fields, and the sum over time cancels to a few percent of its terms' size),
<= 1e-3 on J (a sum of squared residuals: the FP32 traces' ~1e-5 relative
error is amplified where the residual is small).
"""
import numpy as np
import pytest

import oracle
from fdrun import rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl
from paper_1707_03776_gb300.gradient import Propagator, Shot, modelling

pytestmark = pytest.mark.gpu


def _case(seed=3, shape=(28, 24, 32), nt=120):
    h = (10.0,) * 3
    origin = (0.0,) * 3
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    m_true = (1.0 / v ** 2).astype(np.float32)
    g = np.random.default_rng(seed)
    m0 = (m_true * (1.0 + 0.03 * wl.random_field(shape, seed, smooth=2))).astype(np.float32)
    sig = wl.sponge_sigma(shape, h, 5, 2500.0, ref_width=40)
    eta = (m_true.astype(np.float64) * sig).astype(np.float32)
    dt = 0.4 * 10.0 / 2600.0
    src_c = np.array([[60.0, 50.0, 40.0], [200.0, 150.0, 60.0]])
    rec_c = wl.random_points(shape, h, origin, 15, seed + 1, margin=2.0)
    src = np.stack([wl.ricker(nt, dt, 25.0), 0.7 * wl.ricker(nt, dt, 30.0)], axis=1).astype(np.float32)
    _, _, d_obs = oracle.acoustic_forward(shape, h, origin, 8, m_true, eta, dt, nt, src_coords=src_c,
                                          src_trace=src, rec_coords=rec_c, precision="f32")
    return shape, h, origin, m0, eta, dt, src_c, rec_c, src, d_obs.astype(np.float32), nt


def _gpu_gradient(case, k, flags=0):
    import torch
    shape, h, origin, m0, eta, dt, src_c, rec_c, src, d_obs, nt = case
    prop = Propagator(shape, h, origin, 8, Shot(src_c, src, rec_c), nt, dt, checkpoint_every=k, flags=flags)
    prop.set_damping(eta)
    m = torch.from_numpy(m0).cuda().requires_grad_(True)
    rec = modelling(m, prop)
    d = torch.from_numpy(d_obs).cuda()
    loss = 0.5 * ((rec - d) ** 2).sum()
    loss.backward()
    return float(loss.item()), m.grad.detach().cpu().numpy()


def test_gradient_matches_oracle():
    case = _case()
    shape, h, origin, m0, eta, dt, src_c, rec_c, src, d_obs, nt = case
    J, g = _gpu_gradient(case, 25)
    Jo, go = oracle.acoustic_gradient(shape, h, origin, 8, m0.astype(np.float64), eta.astype(np.float64), dt, nt,
                                      src_c, src.astype(np.float64), rec_c, d_obs.astype(np.float64))
    assert abs(J - Jo) <= 1e-3 * Jo, (J, Jo)
    assert rel_l2(g, go) <= 1e-3, rel_l2(g, go)


def test_checkpointing_is_exact():
    """Recomputing segments from checkpoints reproduces the stored-history
    gradient bit for bit (the same kernel on the same inputs), and so does
    keeping the whole forward history (checkpoint_every=0)."""
    case = _case(seed=5, nt=90)
    _, g1 = _gpu_gradient(case, 90)
    _, g2 = _gpu_gradient(case, 17)
    np.testing.assert_array_equal(g1, g2)
    J0, g0 = _gpu_gradient(case, 0)
    np.testing.assert_array_equal(g1, g0)


def test_plain_kernels_agree():
    case = _case(seed=7, nt=60)
    _, g1 = _gpu_gradient(case, 20)
    _, g2 = _gpu_gradient(case, 20, flags=fd.FD_FLAG_PLAIN_KERNELS)
    assert rel_l2(g1, g2) <= 1e-4


def test_step_out_of_place_matches_apply():
    """fd_operator_step between separate buffers equals fd_operator_apply's
    in-place step."""
    import torch
    shape = (20, 30, 70)
    h = (10.0,) * 3
    m = np.full(shape, 1.0 / 2000.0 ** 2, dtype=np.float32)
    u0 = wl.random_field(shape, 1, smooth=1)
    u1 = wl.random_field(shape, 2, smooth=1)
    grid = fd.Grid(shape, h)
    u = fd.TimeData("u", grid)
    md = fd.DenseData("m", grid)
    md.data.copy_(torch.from_numpy(m))
    op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u, md)
    u.at(0).copy_(torch.from_numpy(u0))
    u.at(1).copy_(torch.from_numpy(u1))
    a = torch.zeros_like(u.slots[0])
    b = torch.zeros_like(u.slots[0])
    a[..., :70].copy_(torch.from_numpy(u0))
    b[..., :70].copy_(torch.from_numpy(u1))
    out = torch.zeros_like(u.slots[0])
    fd.fd_operator_step(op.handle, 0, 1e-3, a.data_ptr(), b.data_ptr(), out.data_ptr())
    op.apply(0, 1, 1e-3)
    op.sync()
    np.testing.assert_array_equal(out[..., :70].cpu().numpy(), u.at(1).cpu().numpy())


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_REVERSE, fd.FD_FLAG_PLAIN_KERNELS | fd.FD_FLAG_REVERSE])
def test_fused_imaging_equals_step_then_imaging(flags):
    """fd_operator_apply_imaging (the imaging condition accumulated inside the
    tiled sweep, or after the step on the plain kernels) equals the step
    followed by fd_imaging_accumulate bit for bit, sources included."""
    import torch
    shape = (22, 37, 70)
    h = (10.0,) * 3
    origin = (0.0,) * 3
    nt, n, dt = 6, 3, 1e-3
    m = np.full(shape, 1.0 / 2000.0 ** 2, dtype=np.float32)
    grid = fd.Grid(shape, h, origin)
    src_c = wl.random_points(shape, h, origin, 3, 11, margin=1.0)
    trace = np.random.default_rng(12).standard_normal((nt, 3)).astype(np.float32)
    fields = [torch.zeros(grid.padded_shape, dtype=torch.float32, device="cuda") for _ in range(4)]
    for i, f in enumerate(fields):
        f[..., :shape[2]].copy_(torch.from_numpy(wl.random_field(shape, 20 + i, smooth=1)))
    u0, u1, u2, grad0 = fields
    state = [wl.random_field(shape, 30 + i, smooth=1) for i in range(2)]
    written = n % 2 if flags & fd.FD_FLAG_REVERSE else (n + 1) % 2
    out = []
    for fused in (True, False):
        u = fd.TimeData("u", grid)
        md = fd.DenseData("m", grid)
        md.data.copy_(torch.from_numpy(m))
        src = fd.PointData("src", grid, src_c, nt)
        src.data[:, :3].copy_(torch.from_numpy(trace))
        op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u, md, src=src, flags=flags)
        for s, v in zip(u.slots, state):
            s[..., :shape[2]].copy_(torch.from_numpy(v))
        grad = grad0.clone()
        scale = -1.0 / dt ** 2
        if fused:
            fd.fd_operator_apply_imaging(op.handle, n, dt, scale, u0.data_ptr(), u1.data_ptr(), u2.data_ptr(),
                                         grad.data_ptr())
        else:
            op.apply(n, 1, dt)
            fd.fd_imaging_accumulate(grid.handle, scale, u.slots[written].data_ptr(), u0.data_ptr(), u1.data_ptr(),
                                     u2.data_ptr(), grad.data_ptr(), torch.cuda.current_stream().cuda_stream)
        op.sync()
        torch.cuda.synchronize()
        out.append((u.slots[written][..., :shape[2]].cpu().numpy(), grad[..., :shape[2]].cpu().numpy()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.abs(out[0][1] - grad0[..., :shape[2]].cpu().numpy()).max() > 0


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_imaging_steps_equal_single_passes(k):
    """fd_imaging_accumulate_steps (adjoint steps n .. n-k+1 imaged in one
    pass) equals fd_imaging_accumulate for step n, n-1, ... in turn, bit for
    bit; rows of 37 points take the scalar tail as well."""
    import torch
    shape = (9, 7, 37)
    grid = fd.Grid(shape, (10.0,) * 3)
    f = [torch.zeros(grid.padded_shape, dtype=torch.float32, device="cuda") for _ in range(2 * k + 3)]
    for i, t in enumerate(f):
        t[..., :shape[2]].copy_(torch.from_numpy(wl.random_field(shape, 40 + i, smooth=1)))
    mu, u, g0 = f[:k], f[k:2 * k + 2], f[-1]
    st = torch.cuda.current_stream().cuda_stream
    scale = -1.0 / 1e-3 ** 2
    g1, g2 = g0.clone(), g0.clone()
    for j in range(k):
        fd.fd_imaging_accumulate(grid.handle, scale, mu[j].data_ptr(), u[j].data_ptr(), u[j + 1].data_ptr(),
                                 u[j + 2].data_ptr(), g1.data_ptr(), st)
    fd.fd_imaging_accumulate_steps(grid.handle, scale, [t.data_ptr() for t in mu], [t.data_ptr() for t in u],
                                   g2.data_ptr(), st)
    torch.cuda.synchronize()
    n2 = shape[2]
    assert torch.equal(g1[..., :n2], g2[..., :n2])
    assert not torch.equal(g2[..., :n2], g0[..., :n2])
    with pytest.raises(fd.FDError):
        fd.fd_imaging_accumulate_steps(grid.handle, scale, [t.data_ptr() for t in mu], [t.data_ptr() for t in u],
                                       u[0].data_ptr(), st)


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS])
def test_grouped_backward_equals_per_step_imaging(flags):
    """Where the sweep does not inject the residual itself, the backward sweep
    runs up to four adjoint steps out of place and images them in one pass.
    Its gradient equals the per-step loop (fd_operator_apply_imaging at every
    step, in the operator's own slots) bit for bit; 61 steps leave a last group
    of fewer than four."""
    import torch
    case = _case(seed=7, nt=61)
    shape, h, origin, m0, eta, dt, src_c, rec_c, src, d_obs, nt = case
    prop = Propagator(shape, h, origin, 8, Shot(src_c, src, rec_c), nt, dt, checkpoint_every=0, flags=flags)
    prop.set_damping(eta)
    prop.set_model(torch.from_numpy(m0).cuda())
    residual = prop.forward().clone() - torch.from_numpy(d_obs).cuda()
    g_grouped = prop.backward(residual).clone()
    for s in prop.mu.slots:
        s.zero_()
    prop.grad.slots[0].zero_()
    scale = -1.0 / dt ** 2
    gp = prop.grad.slots[0].data_ptr()
    hist = prop.hist
    for n in range(nt - 1, -1, -1):
        if n >= 1:
            fd.fd_operator_apply_imaging(prop.adj.handle, n, dt, scale, hist[n + 1].data_ptr(), hist[n].data_ptr(),
                                         hist[n - 1].data_ptr(), gp)
        else:
            prop.adj.apply(n, 1, dt)
    prop.adj.sync()
    if flags & fd.FD_FLAG_PLAIN_KERNELS:
        assert not fd.fd_operator_sources_fused(prop.adj.handle)
    assert torch.equal(g_grouped, prop.grad.data)
    assert float(g_grouped.abs().max()) > 0


def test_receiver_lattice_is_injected_inside_the_chunked_sweep():
    """The adjoint's sources are a receiver lattice: thousands of corners in
    the tile columns at the receivers' depth.  On a grid small enough that the
    planner splits d0 into chunks, each chunk's CTA stages only its own planes'
    corners, so the sweep injects them itself (fd_operator_sources_fused) and
    apply_imaging fuses the imaging condition.  Eight adjoint steps with imaging
    then agree with the plain kernels (atomic injection, separate imaging) to
    FP32 rounding (the injection sums round in another order)."""
    import torch
    shape = (96, 96, 96)
    h = (10.0,) * 3
    origin = (0.0,) * 3
    nt, dt = 8, 1e-3
    g = np.random.default_rng(77)
    side = np.linspace(50.0, 900.0, 33)
    X, Y = np.meshgrid(side, side, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 105.0)], axis=1)
    trace = g.standard_normal((nt, rec.shape[0])).astype(np.float32)
    m = (1.0 / wl.random_smooth_velocity(shape, 5, sigma_cells=6.0, vmin=1800.0, vmax=2600.0) ** 2).astype(np.float32)
    grid = fd.Grid(shape, h, origin)
    hist = [torch.zeros(grid.padded_shape, dtype=torch.float32, device="cuda") for _ in range(nt + 2)]
    for i, f in enumerate(hist):
        f[..., :shape[2]].copy_(torch.from_numpy(wl.random_field(shape, 40 + i, smooth=1)))
    results = []
    for flags in (fd.FD_FLAG_REVERSE, fd.FD_FLAG_REVERSE | fd.FD_FLAG_PLAIN_KERNELS):
        mu = fd.TimeData("mu", grid)
        md = fd.DenseData("m", grid)
        md.data.copy_(torch.from_numpy(m))
        src = fd.PointData("res", grid, rec, nt)
        src.data[:, : rec.shape[0]].copy_(torch.from_numpy(trace))
        op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, mu, md, src=src, flags=flags)
        if not flags & fd.FD_FLAG_PLAIN_KERNELS:
            rows, stages, ctas = fd.fd_operator_get_tiling(op.handle)
            columns = -(-shape[1] // rows) * -(-shape[2] // 64)
            assert ctas > columns, (rows, ctas, columns)  # d0 chunks
            assert fd.fd_operator_sources_fused(op.handle)
        else:
            assert not fd.fd_operator_sources_fused(op.handle)
        grad = torch.zeros_like(hist[0])
        for n in range(nt - 1, -1, -1):
            fd.fd_operator_apply_imaging(op.handle, n, dt, -1.0 / dt ** 2, hist[n].data_ptr(), hist[n + 1].data_ptr(),
                                         hist[n + 2].data_ptr(), grad.data_ptr())
        op.sync()
        torch.cuda.synchronize()
        results.append((mu.slots[0][..., :shape[2]].cpu().numpy().astype(np.float64),
                        grad[..., :shape[2]].cpu().numpy().astype(np.float64)))
    (ua, ga), (ub, gb) = results
    assert np.abs(ga).max() > 0
    assert np.linalg.norm(ua - ub) <= 1e-6 * np.linalg.norm(ub)
    assert np.linalg.norm(ga - gb) <= 1e-6 * np.linalg.norm(gb)
