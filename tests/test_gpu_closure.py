"""Learned closure on the GPU against the CPU oracle (oracle/cnn.py).

Operands are BF16 on both sides (the oracle takes the BF16-rounded inputs and
weights in FP64), so the convolution's only difference is the GPU's FP32
accumulation over K = 27 taps x 16 channels: |gpu - ref| <= 2e-5 * A, with A
the same sum taken over absolute values (K * 2^-24 ~ 2.6e-5 bounds the
relative error of a K-term FP32 sum; the tensor cores' accumulation stays
within it).  BF16 outputs add one rounding: 2^-8 |ref|.  The whole network
stores every activation and gradient in BF16; against the oracle storing
them the same way only the accumulation order differs (relative L2 2e-3),
against the exact FP64 network the BF16 storage costs up to ~3 % at the first
layer's weight gradient (6e-2 allowed).

Shapes span several CTA tiles in every direction with ragged ends (tiles of
16 planes x 8 rows x 64 points).
"""
import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu

SHAPE = (20, 19, 70)


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _fd():
    from paper_1707_03776_gb300 import fd
    return fd


def _bf16_acts(x16):
    """numpy [N..., 16] -> (device BF16 tensor [Npts, 16], the BF16 values in FP64)."""
    torch = _torch()
    xr = cnn.bf16_round(np.asarray(x16, dtype=np.float32))
    t = torch.from_numpy(xr.reshape(-1, 16)).to(torch.bfloat16).cuda()
    return t, xr.astype(np.float64)


def _pad16(x):
    out = np.zeros(x.shape[:3] + (16,), dtype=x.dtype)
    out[..., : x.shape[3]] = x
    return out


def _pack(w, flip=0):
    torch = _torch()
    fd = _fd()
    cin, cout = w.shape[1], w.shape[2]
    n = cin if flip else cout
    frag = torch.zeros(27 * ((n + 7) // 8) * 256, dtype=torch.uint8, device="cuda")
    wd = torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
    fd.fd_cnn_pack_weights(wd, cin, cout, flip, frag, torch.cuda.current_stream().cuda_stream)
    return frag, cnn.bf16_round(w.astype(np.float32)).astype(np.float64)


@pytest.mark.parametrize("cin,cout,relu,mask", [(6, 16, True, False), (16, 16, False, True), (16, 5, True, True),
                                                (3, 8, False, False)])
def test_conv3d_parity(cin, cout, relu, mask):
    torch = _torch()
    fd = _fd()
    g = np.random.default_rng(100 + cin + cout)
    x = _pad16(g.standard_normal(SHAPE + (cin,)).astype(np.float32))
    w = (g.standard_normal((27, cin, cout)) / np.sqrt(27 * cin)).astype(np.float32)
    b = g.standard_normal(cout).astype(np.float32)
    xt, xr = _bf16_acts(x)
    frag, wr = _pack(w)
    bt = torch.from_numpy(b).cuda()
    mk = g.standard_normal(SHAPE + (16,)).astype(np.float32)
    mt, mr = _bf16_acts(mk)
    y = torch.full((xt.shape[0], 16), float("nan"), dtype=torch.bfloat16, device="cuda")
    fd.fd_cnn_conv3d(SHAPE, xt, frag, bt, cout, int(relu), mt if mask else None, y, 0,
                     torch.cuda.current_stream().cuda_stream)
    got = y.float().cpu().numpy().reshape(SHAPE + (16,)).astype(np.float64)
    ref = cnn.conv3d(xr[..., :cin], wr, b.astype(np.float64))
    A = cnn.conv3d(np.abs(xr[..., :cin]), np.abs(wr), np.abs(b.astype(np.float64)))
    if relu:
        ref = np.maximum(ref, 0.0)
    if mask:
        ref = ref * (mr[..., :cout] > 0)
    tol = 2.0 ** -8 * np.abs(ref) + 2e-5 * A
    assert np.all(np.abs(got[..., :cout] - ref) <= tol + 1e-30)
    assert np.all(got[..., cout:] == 0.0)  # channels beyond cout are written as zero


def test_conv3d_fp32_output_parity():
    torch = _torch()
    fd = _fd()
    g = np.random.default_rng(7)
    x = g.standard_normal(SHAPE + (16,)).astype(np.float32)
    w = (g.standard_normal((27, 16, 1)) / 20.0).astype(np.float32)
    xt, xr = _bf16_acts(x)
    frag, wr = _pack(w)
    y = torch.zeros(xt.shape[0], dtype=torch.float32, device="cuda")
    fd.fd_cnn_conv3d(SHAPE, xt, frag, None, 1, 0, None, y, 1, torch.cuda.current_stream().cuda_stream)
    got = y.cpu().numpy().reshape(SHAPE).astype(np.float64)
    ref = cnn.conv3d(xr, wr, np.zeros(1))[..., 0]
    A = cnn.conv3d(np.abs(xr), np.abs(wr), np.zeros(1))[..., 0]
    assert np.all(np.abs(got - ref) <= 2e-5 * A + 1e-30)


@pytest.mark.parametrize("cin,cout", [(16, 1), (16, 16), (6, 16)])
def test_conv3d_input_gradient_parity(cin, cout):
    """The flipped pack turns the convolution into its input gradient."""
    torch = _torch()
    fd = _fd()
    g = np.random.default_rng(200 + cin + cout)
    gy = _pad16(g.standard_normal(SHAPE + (cout,)).astype(np.float32))
    w = (g.standard_normal((27, cin, cout)) / np.sqrt(27 * cout)).astype(np.float32)
    gt, gr = _bf16_acts(gy)
    frag, wr = _pack(w, flip=1)
    y = torch.zeros((gt.shape[0], 16), dtype=torch.bfloat16, device="cuda")
    fd.fd_cnn_conv3d(SHAPE, gt, frag, None, cin, 0, None, y, 0, torch.cuda.current_stream().cuda_stream)
    got = y.float().cpu().numpy().reshape(SHAPE + (16,)).astype(np.float64)
    ref = cnn.conv3d_grad_input(gr[..., :cout], wr)
    A = cnn.conv3d_grad_input(np.abs(gr[..., :cout]), np.abs(wr))
    assert np.all(np.abs(got[..., :cin] - ref) <= 2.0 ** -8 * np.abs(ref) + 2e-5 * A + 1e-30)


@pytest.mark.parametrize("cin,cout", [(16, 16), (6, 16), (16, 1)])
def test_conv3d_weight_gradient_parity(cin, cout):
    torch = _torch()
    fd = _fd()
    g = np.random.default_rng(300 + cin + cout)
    x = _pad16(g.standard_normal(SHAPE + (cin,)).astype(np.float32))
    gy = _pad16(g.standard_normal(SHAPE + (cout,)).astype(np.float32))
    xt, xr = _bf16_acts(x)
    gt, gr = _bf16_acts(gy)
    gw = torch.full((27, cin, cout), 0.25, dtype=torch.float32, device="cuda")  # accumulates onto 0.25
    gb = torch.zeros(16, dtype=torch.float32, device="cuda")
    fd.fd_cnn_conv3d_wgrad(SHAPE, xt, gt, cin, cout, gw, gb, torch.cuda.current_stream().cuda_stream)
    rw, rb = cnn.conv3d_grad_weight(xr[..., :cin], gr[..., :cout])
    Aw, Ab = cnn.conv3d_grad_weight(np.abs(xr[..., :cin]), np.abs(gr[..., :cout]))
    got = gw.cpu().numpy().astype(np.float64) - 0.25
    assert np.all(np.abs(got - rw) <= 2e-5 * Aw + 1e-6)
    assert np.all(np.abs(gb.cpu().numpy()[:cout] - rb) <= 2e-5 * Ab + 1e-6)


def _grid_fields(shape, seed):
    torch = _torch()
    fd = _fd()
    g = np.random.default_rng(seed)
    grid = fd.Grid(shape, (20.0,) * 3)
    u = fd.TimeData("u", grid)
    m = fd.DenseData("m", grid)
    un, up = g.standard_normal(shape).astype(np.float32), g.standard_normal(shape).astype(np.float32)
    v = g.uniform(1500.0, 3500.0, shape)
    mm = (1.0 / v ** 2).astype(np.float32)
    u.view(0).copy_(torch.from_numpy(un))
    u.view(1).copy_(torch.from_numpy(up))
    m.data.copy_(torch.from_numpy(mm))
    return grid, u, m, un, up, mm


def test_features_restrict_correction_mse_adam():
    torch = _torch()
    fd = _fd()
    st = torch.cuda.current_stream().cuda_stream
    shape = (9, 10, 13)
    grid, u, m, un, up, mm = _grid_fields(shape, 5)
    n = int(np.prod(shape))
    x = torch.full((n, 16), float("nan"), dtype=torch.bfloat16, device="cuda")
    fd.fd_cnn_features(grid.handle, u.slots[0], u.slots[1], m.slots[0], 2.0, 3000.0, x, st)
    ref = cnn.features(un, up, mm, 2.0, 3000.0)
    got = x.float().cpu().numpy().reshape(shape + (16,))
    assert np.all(np.abs(got[..., :6] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(ref).max())
    assert np.all(got[..., 6:] == 0.0)
    # the training-time noise: SplitMix64 deviates on both sides
    fd.fd_cnn_features(grid.handle, u.slots[0], u.slots[1], m.slots[0], 2.0, 3000.0, x, st, noise=0.3, seed=777)
    nu, nup = cnn.noisy_states(un, up, 0.3, 777)
    ref = cnn.features(nu, nup, mm, 2.0, 3000.0)
    got = x.float().cpu().numpy().reshape(shape + (16,))
    assert np.all(np.abs(got[..., :6] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    # with three model descriptors: channels 6..11, the rest zero
    from paper_1707_03776_gb300 import workloads as wl
    subs = [wl.random_field(shape, 60 + k) for k in range(3)]
    sub = torch.zeros((3,) + grid.padded_shape, dtype=torch.float32, device="cuda")
    for k in range(3):
        sub[k, ..., : shape[2]].copy_(torch.from_numpy(subs[k]))
    x.fill_(float("nan"))
    fd.fd_cnn_features_sub(grid.handle, u.slots[0], u.slots[1], m.slots[0], sub, 3, 2.0, 3000.0, x, st)
    ref = cnn.features(un, up, mm, 2.0, 3000.0, sub=subs)
    got = x.float().cpu().numpy().reshape(shape + (16,))
    assert np.all(np.abs(got[..., :12] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(ref).max())
    assert np.all(got[..., 12:] == 0.0)

    # restriction from a (2n-1)-node fine grid, with the sum of squares
    fshape = tuple(2 * s - 1 for s in shape)
    fgrid = fd.Grid(fshape, (10.0,) * 3)
    fu = fd.DenseData("f", fgrid)
    fine = np.random.default_rng(6).standard_normal(fshape).astype(np.float32)
    fu.data.copy_(torch.from_numpy(fine))
    out = fd.DenseData("c", grid)
    ss = torch.zeros(1, dtype=torch.float32, device="cuda")
    fd.fd_cnn_restrict(fgrid.handle, fu.slots[0], grid.handle, out.slots[0], 2, ss, st)
    r = cnn.restrict(fine, 2)
    assert np.array_equal(out.data.cpu().numpy(), r)
    assert abs(float(ss.item()) - float((r.astype(np.float64) ** 2).sum())) <= 1e-5 * float((r ** 2).sum())
    with pytest.raises(fd.FDError):
        fd.fd_cnn_restrict(fgrid.handle, fu.slots[0], grid.handle, out.slots[0], 3, None, st)

    # u += scale * corr
    corr = np.random.default_rng(8).standard_normal(n).astype(np.float32)
    fd.fd_cnn_add_correction(grid.handle, u.slots[0], torch.from_numpy(corr).cuda(), 0.5, st)
    np.testing.assert_allclose(u.view(0).cpu().numpy(), un + np.float32(0.5) * corr.reshape(shape), rtol=1e-6,
                               atol=1e-6)

    # loss and gradient against (target - base)/s
    pred = np.random.default_rng(9).standard_normal(n).astype(np.float32)
    gy = torch.zeros((n, 16), dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    tgt, base = fd.DenseData("t", grid), fd.DenseData("b", grid)
    tv = np.random.default_rng(10).standard_normal(shape).astype(np.float32)
    bv = np.random.default_rng(11).standard_normal(shape).astype(np.float32)
    tgt.data.copy_(torch.from_numpy(tv))
    base.data.copy_(torch.from_numpy(bv))
    fd.fd_cnn_mse_grad(grid.handle, torch.from_numpy(pred).cuda(), tgt.slots[0], base.slots[0], 4.0, gy, loss, st)
    rl, rg = cnn.mse_and_grad(pred.reshape(shape), (tv.astype(np.float64) - bv) / 4.0)
    assert abs(float(loss.item()) - rl) <= 1e-5 * rl
    gg = gy.float().cpu().numpy().reshape(shape + (16,))
    assert np.all(np.abs(gg[..., 0] - rg) <= 2.0 ** -8 * np.abs(rg) + 1e-12)
    assert np.all(gg[..., 1:] == 0.0)

    # Adam, three steps
    g = np.random.default_rng(12)
    p = g.standard_normal(1000)
    pt = torch.from_numpy(p.astype(np.float32)).cuda()
    m1 = torch.zeros_like(pt)
    m2 = torch.zeros_like(pt)
    rp, rm1, rm2 = p.astype(np.float32).astype(np.float64), np.zeros(1000), np.zeros(1000)
    for step in (1, 2, 3):
        gr = g.standard_normal(1000).astype(np.float32)
        fd.fd_cnn_adam(pt, torch.from_numpy(gr).cuda(), m1, m2, 1000, 1e-3, 0.9, 0.999, 1e-8, step, st)
        rp, rm1, rm2 = cnn.adam(rp, gr.astype(np.float64), rm1, rm2, 1e-3, 0.9, 0.999, 1e-8, step)
    np.testing.assert_allclose(pt.cpu().numpy(), rp, rtol=0, atol=1e-6)


def test_network_gradients_parity():
    """Forward, loss and backward of the whole closure network (closure.py on
    libfdgb) against the oracle's network on the same BF16 weights and
    features."""
    torch = _torch()
    fd = _fd()
    from paper_1707_03776_gb300 import closure
    st = torch.cuda.current_stream().cuda_stream
    shape = (18, 11, 67)
    grid, u, m, un, up, mm = _grid_fields(shape, 21)
    net = closure.ClosureNet(seed=3, rho=1.0)
    ws = closure.Workspace(shape)
    fd.fd_cnn_features(grid.handle, u.slots[0], u.slots[1], m.slots[0], 1.5, net.vref, ws.h[0], st)
    closure.network_forward(net, ws, st)
    tgt, base = fd.DenseData("t", grid), fd.DenseData("b", grid)
    tv = np.random.default_rng(22).standard_normal(shape).astype(np.float32)
    tgt.data.copy_(torch.from_numpy(tv))
    net.grads.zero_()
    fd.fd_cnn_mse_grad(grid.handle, ws.out, tgt.slots[0], None, 1.5, ws.g[0], ws.loss, st)
    closure.network_backward(net, ws, st)

    ws_np = [cnn.bf16_round(w).astype(np.float64) for w in net.weights()]
    params = [(w, np.zeros(w.shape[2])) for w in ws_np]
    x = cnn.bf16_round(cnn.features(un, up, mm, 1.5, net.vref).astype(np.float32)).astype(np.float64)
    out = ws.out.cpu().numpy().reshape(shape)
    got = [net.grad(li).cpu().numpy() for li in range(4)]
    # (1) the oracle storing activations and gradients in BF16 like the
    # device: only accumulation order differs
    acts, pre = cnn.network_forward(x, params, store=cnn.bf16_round)
    loss_b, gout = cnn.mse_and_grad(acts[-1][..., 0], tv / 1.5)
    assert np.linalg.norm(out - acts[-1][..., 0]) <= 1e-3 * np.linalg.norm(acts[-1])
    assert abs(float(ws.loss.item()) - loss_b) <= 1e-4 * loss_b
    grads = cnn.network_backward(acts, pre, params, gout[..., None], store=cnn.bf16_round)
    for li in range(4):
        assert np.linalg.norm(got[li] - grads[li][0]) <= 2e-3 * np.linalg.norm(grads[li][0]), li
    # (2) the exact FP64 network's output: the device stores three BF16
    # activations on the way (unit roundoff 2^-9 each), so its output stays
    # within 1e-2 of the unrounded network.  The gradients are judged by (1)
    # only: with BF16 storage of both activations and gradients their
    # distance to the unrounded network measures BF16, not the kernels.
    acts, pre = cnn.network_forward(x, params)
    assert np.linalg.norm(out - acts[-1][..., 0]) <= 1e-2 * np.linalg.norm(acts[-1])


def test_closure_step_parity():
    """One step of the closure operator = the oracle's coarse step from the
    same state plus rho times the oracle network on the same weights."""
    torch = _torch()
    import oracle
    from paper_1707_03776_gb300 import closure, workloads as wl
    cfg = wl.closure_config(n_coarse=24, nt=40, seed=4, sponge=4)
    c = cfg["coarse"]
    net = closure.ClosureNet(seed=5, rho=0.01)
    op = closure.ClosureOperator(cfg, net)
    # 30 learned steps on the GPU, then the 31st step's pieces one by one
    # from the GPU's state
    op.run(30)
    uc = op.u.view(30 % 2).cpu().numpy().copy()
    upv = op.u.view(31 % 2).cpu().numpy().copy()
    from paper_1707_03776_gb300 import fd
    st = torch.cuda.current_stream().cuda_stream
    fd.fd_cnn_features(op.grid.handle, op.u.slots[30 % 2], op.u.slots[31 % 2], op.m.slots[0], 1.0, net.vref,
                       op.ws.h[0], st)
    closure.network_forward(net, op.ws, st)
    op.op.apply(30, 1, op.dt)
    fd.fd_cnn_add_correction(op.grid.handle, op.u.slots[31 % 2], op.ws.out, net.rho, st)
    got = op.u.view(31 % 2).cpu().numpy()

    nxt, _, _ = oracle.acoustic_forward(c["shape"], c["spacing"], cfg["origin"], 4, c["m"], c["eta"], c["dt"], 1,
                                        src_coords=c["src_coords"], src_trace=c["src_trace"], u_cur=uc,
                                        u_prev=upv, t0=30, n_total=c["nt"])
    params = [(cnn.bf16_round(w).astype(np.float64), np.zeros(w.shape[2])) for w in net.weights()]
    corr = cnn.closure_correction(uc, upv, c["m"], params, net.rho, net.vref)
    ref = nxt + corr
    # the coarse step agrees to FP32 rounding; the correction to BF16 activations
    err = np.linalg.norm(got - ref)
    assert err <= 1e-5 * np.linalg.norm(nxt) + 2e-2 * np.linalg.norm(corr)
    assert np.linalg.norm(corr) > 0


def test_closure_rollout_parity():
    """40 learned steps from rest on the GPU against the oracle's coarse steps
    plus the oracle network's correction (FP64 network on the same BF16
    weights).  The correction is ~rho of the field, so its BF16 storage error
    is ~1e-2 of rho relative: the traces agree to 1e-4."""
    torch = _torch()
    import oracle
    from paper_1707_03776_gb300 import closure, workloads as wl
    cfg = wl.closure_config(n_coarse=20, nt=40, seed=9, sponge=3, src_sigma=25.0)
    c = cfg["coarse"]
    net = closure.ClosureNet(seed=7, rho=0.01)
    op = closure.ClosureOperator(cfg, net)
    got = op.run(40).cpu().numpy().copy()
    params = [(cnn.bf16_round(w).astype(np.float64), np.zeros(w.shape[2])) for w in net.weights()]
    uc = np.zeros(c["shape"])
    up = np.zeros(c["shape"])
    rec = np.zeros_like(got, dtype=np.float64)
    for n in range(40):
        corr = cnn.closure_correction(uc, up, c["m"], params, net.rho, net.vref)
        nxt, _, tr = oracle.acoustic_forward(c["shape"], c["spacing"], cfg["origin"], 4, c["m"], c["eta"], c["dt"],
                                             1, src_coords=c["src_coords"], src_trace=c["src_trace"],
                                             rec_coords=cfg["rec_coords"], u_cur=uc, u_prev=up, t0=n,
                                             n_total=c["nt"])
        rec[n] = tr[n]
        up, uc = uc, nxt + corr
    assert np.linalg.norm(got - rec) <= 1e-4 * np.linalg.norm(rec)
    plain = op.run(40, learned=False).cpu().numpy()
    assert np.linalg.norm(plain - rec) > 10 * np.linalg.norm(got - rec)  # the correction is visible


def test_training_lowers_loss_and_trace_error():
    """Training on 32 layered-model runs lowers the one-step loss tenfold, and the
    trained closure's receiver traces are closer to the fine grid's than the
    plain coarse run's on an unseen model of the training configuration (8-cell
    sponge; smaller than the evaluation workload).  This checks that training
    works end to end on the GPU kernels; the gain it measures lies mostly in
    the boundary region (bench.py's learned row also compares with a 24-cell
    sponge, where it vanishes)."""
    _torch()
    from paper_1707_03776_gb300 import closure, workloads as wl
    net, data, hist = closure.train_default(count=32, n_coarse=64, nt=600, iters=800, log_every=100)
    # first entry: the untrained network's loss; last: the mean of the last 100
    assert hist[-1][1] < 0.1 * hist[0][1], hist
    cfg = wl.closure_config(64, 800, seed=1000, src="surface")
    ref = closure.FineReference(cfg).run().cpu().numpy()
    op = closure.ClosureOperator(cfg, net)
    plain = closure.trace_error(op.run(learned=False).cpu().numpy(), ref)
    learned = closure.trace_error(op.run(learned=True).cpu().numpy(), ref)
    assert np.isfinite(learned) and learned < 0.85 * plain, (learned, plain)


@pytest.mark.parametrize("cin,cout,relu,mask,flip,f32,shape", [
    (6, 16, True, False, 0, False, (19, 7, 150)), (16, 16, False, True, 0, False, (19, 7, 150)),
    (16, 5, True, True, 0, False, (19, 7, 150)), (16, 1, False, False, 0, True, (19, 7, 150)),
    (16, 16, False, True, 1, False, (19, 7, 150)), (6, 16, False, False, 1, False, (19, 7, 150)),
    (16, 16, True, False, 0, False, (70, 6, 260)), (16, 16, True, False, 0, False, (64, 17, 128)),
    (6, 16, True, False, 0, False, (1, 1, 1))])
def test_conv3d_tensor_memory_path(cin, cout, relu, mask, flip, f32, shape):
    """The tcgen05 kernel against the oracle (BF16 operands, exact sums) and
    against the mma.sync kernel: both accumulate in FP32, the tcgen05 one as
    two tap halves added at the end, so the two differ by FP32 rounding --
    at most one BF16 rounding step of the stored outputs, and 1e-6 relative
    for the FP32 channel.  Shapes ragged against its 2-row x 128-point tile
    columns, with one (tile column, plane) item per CTA and with CTA shares
    of several planes that cross tile columns."""
    torch = _torch()
    fd = _fd()
    st = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(400 + cin + cout + flip)
    nin = cout if flip else cin  # channels the convolution reads
    nout = cin if flip else cout
    x = _pad16(g.standard_normal(shape + (nin,)).astype(np.float32))
    w = (g.standard_normal((27, cin, cout)) / np.sqrt(27 * nin)).astype(np.float32)
    xt, xr = _bf16_acts(x)
    mt, mr = _bf16_acts(g.standard_normal(shape + (16,)).astype(np.float32))
    wd = torch.from_numpy(w).cuda()
    frag = torch.zeros(27 * 512, dtype=torch.uint8, device="cuda")
    frag_tc = torch.zeros(27 * 512, dtype=torch.uint8, device="cuda")
    fd.fd_cnn_pack_weights(wd, cin, cout, flip, frag, st)
    fd.fd_cnn_pack_weights_tc(wd, cin, cout, flip, frag_tc, st)
    n = xt.shape[0]
    mk = mt if mask else None
    if f32:
        y1 = torch.zeros(n, dtype=torch.float32, device="cuda")
        y2 = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    else:
        y1 = torch.zeros((n, 16), dtype=torch.bfloat16, device="cuda")
        y2 = torch.full((n, 16), float("nan"), dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    fd.fd_cnn_conv3d(shape, xt, frag, None, nout, int(relu), mk, y1, int(f32), st)
    fd.fd_cnn_conv3d_tc(shape, xt, frag_tc, None, nout, int(relu), mk, y2, int(f32), status, st)
    torch.cuda.synchronize()
    assert status.item() == 0
    a1, a2 = y1.float().cpu().numpy(), y2.float().cpu().numpy()
    assert np.isfinite(a2).all()
    if f32:
        assert np.abs(a2 - a1).max() <= 1e-6 * np.abs(a1).max()
    else:
        # one BF16 step (at most 2^-7 relative) where the FP32 sums round apart, and
        # near zero the FP32 rounding of the sum itself (its terms are up to
        # the outputs' size)
        bound = 2.0 ** -7 * np.abs(a1) + 1e-4 * np.abs(a1).max()
        assert (np.abs(a2 - a1) <= bound).all(), np.abs(a2 - a1).max()
    wr = cnn.bf16_round(w).astype(np.float64)
    ref = cnn.conv3d_grad_input(xr[..., :cout], wr) if flip else cnn.conv3d(xr[..., :cin], wr, np.zeros(cout))
    if relu:
        ref = np.maximum(ref, 0.0)
    if mask:
        ref = ref * (mr[..., :nout] > 0)
    if f32:
        got = y2.cpu().numpy().reshape(shape)
        ref = ref[..., 0]
    else:
        got = y2.float().cpu().numpy().reshape(shape + (16,))[..., :nout]
    assert np.abs(got - ref).max() <= 2.0 ** -8 * np.abs(ref).max() + 1e-4 * np.abs(ref).max()


def test_conv3d_rejects_misaligned_buffers():
    """The 16-byte input copies need a 16-byte aligned x: checked on the host."""
    torch = _torch()
    fd = _fd()
    st = torch.cuda.current_stream().cuda_stream
    shape = (4, 4, 4)
    buf = torch.zeros((64 * 16 + 8,), dtype=torch.bfloat16, device="cuda")
    frag = torch.zeros(27 * 512, dtype=torch.uint8, device="cuda")
    y = torch.zeros((64, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(fd.FDError) as e:
        fd.fd_cnn_conv3d(shape, buf.data_ptr() + 2, frag, None, 16, 0, None, y, 0, st)
    assert e.value.status == fd.FD_ERR_LAYOUT
