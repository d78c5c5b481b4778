"""Learned closure: a coarse-grid acoustic operator corrected at every step by
a small 3D CNN trained on the fine-grid operator's own wavefields.

The coarse update (20 m, SO4) misses the fine one (10 m, SO16) by a local
truncation error that depends on the wavefield near each node and on the
velocity.  Given the coarse states u^n, u^{n-1} (features: u, du, q u, q du,
q^2 u, q^2 du with du = u^n - u^{n-1}, q = 1/(m vref^2)), the network predicts
the one-step residual
    r^n = R u_f^{n+1} - S_c(R u_f^n, R u_f^{n-1})
(R: injection of the fine grid's nodes that coincide with coarse nodes, S_c:
the coarse operator's step, source included), and inference adds it back:
    u^{n+1} = S_c(u^n, u^{n-1}) + rho * CNN(features(u^n, u^{n-1})).
The network has no biases, so it is positively homogeneous in the wavefield
like the residual it learns (the wave equation is linear): training
normalises every sample by its own RMS and inference needs no scale.

Layers: conv3x3x3(6 -> 16) ReLU, (16 -> 16) ReLU, (16 -> 16) ReLU, (16 -> 1);
BF16 weights and activations, FP32 accumulation (libfdgb's fd_cnn_* tensor-
core kernels: the tcgen05 convolution by default, the mma.sync one -- equal
to FP32 rounding, half as fast -- as the alternative);
FP32 master weights updated by Adam.  Every step of training and inference
runs in libfdgb's kernels; torch supplies device memory.
"""
import math

import numpy as np

from . import fd

CHANNELS = (6, 16, 16, 16, 1)
NLAYER = len(CHANNELS) - 1
# model descriptors a network built with nsub > 0 reads (workloads.closure_descriptors)
MAX_SUB = 3


def channels(nsub=0, hidden=3):
    """Channel counts of the layers: 6 wavefield features plus 2 per model
    descriptor in, then `hidden` layers of 16 channels, then 1."""
    return (6 + 2 * int(nsub),) + (16,) * int(hidden) + (1,)
# convolutions on the tcgen05 kernel (fd_cnn_conv3d_tc) unless a caller asks
# for the mma.sync one (fd_cnn_conv3d); they agree to FP32 rounding
TENSOR_MEMORY = True


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _frag_bytes(n):
    return 27 * ((n + 7) // 8) * 256


class ClosureNet:
    """FP32 master weights w[l] [27, cin, cout] (one flat buffer, so that one
    Adam launch updates all) and their packed BF16 tensor-core operands: frag
    (forward) and frag_t (input gradient, taps mirrored) per layer.  With
    nsub > 0 the first layer also reads (s_k u, s_k du) for the first nsub
    model descriptors s_k."""

    def __init__(self, seed=0, rho=1.0, nsub=0, hidden=3):
        import torch
        self.torch = torch
        if not 0 <= int(nsub) <= MAX_SUB:
            raise ValueError("nsub must be in 0..%d" % MAX_SUB)
        if int(hidden) < 1:
            raise ValueError("hidden must be >= 1")
        self.nsub = int(nsub)
        self.channels = channels(nsub, hidden)
        self.nlayer = len(self.channels) - 1
        CH = self.channels
        L = self.nlayer
        sizes = [27 * CH[i] * CH[i + 1] for i in range(L)]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        n = int(self.offsets[-1])
        g = np.random.default_rng(seed)
        init = []
        for li in range(L):
            cin = CH[li]
            std = math.sqrt(2.0 / (27 * cin)) * (0.1 if li == L - 1 else 1.0)
            init.append(g.standard_normal(sizes[li]) * std)
        self.params = torch.from_numpy(np.concatenate(init).astype(np.float32)).cuda()
        self.grads = torch.zeros(n, dtype=torch.float32, device="cuda")
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.adam_step = 0
        self.gb_dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
        self.frag = [torch.zeros(_frag_bytes(CH[i + 1]), dtype=torch.uint8, device="cuda")
                     for i in range(L)]
        self.frag_t = [torch.zeros(_frag_bytes(CH[i]), dtype=torch.uint8, device="cuda")
                       for i in range(L)]
        # tcgen05 operand layout of the same weights, forward and mirrored
        self.frag_tc = [torch.zeros(27 * 512, dtype=torch.uint8, device="cuda") for _ in range(L)]
        self.frag_tc_t = [torch.zeros(27 * 512, dtype=torch.uint8, device="cuda") for _ in range(L)]
        self.tc_status = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.rho = float(rho)
        self.vref = 3500.0
        self.pack()

    def weight(self, li):
        a, b = int(self.offsets[li]), int(self.offsets[li + 1])
        return self.params[a:b].view(27, self.channels[li], self.channels[li + 1])

    def grad(self, li):
        a, b = int(self.offsets[li]), int(self.offsets[li + 1])
        return self.grads[a:b].view(27, self.channels[li], self.channels[li + 1])

    def pack(self):
        st = _stream()
        for li in range(self.nlayer):
            cin, cout = self.channels[li], self.channels[li + 1]
            fd.fd_cnn_pack_weights(self.weight(li), cin, cout, 0, self.frag[li], st)
            fd.fd_cnn_pack_weights_tc(self.weight(li), cin, cout, 0, self.frag_tc[li], st)
            if li > 0:
                fd.fd_cnn_pack_weights(self.weight(li), cin, cout, 1, self.frag_t[li], st)
                fd.fd_cnn_pack_weights_tc(self.weight(li), cin, cout, 1, self.frag_tc_t[li], st)

    def check(self):
        """Raise if a tcgen05 convolution gave up on a bounded wait (the
        status word its kernels write; reading it synchronises)."""
        code = int(self.tc_status.item())
        if code != 0:
            self.tc_status.zero_()
            raise fd.FDError(code, "a tcgen05 convolution gave up on a bounded wait")

    def set_weights(self, ws):
        """Load FP32 weights [(27, cin, cout)] per layer (numpy) and repack."""
        for li, w in enumerate(ws):
            self.weight(li).copy_(self.torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)))
        self.pack()

    def weights(self):
        return [self.weight(li).cpu().numpy().copy() for li in range(self.nlayer)]

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.adam_step += 1
        fd.fd_cnn_adam(self.params, self.grads, self.m1, self.m2, self.params.numel(), lr, beta1, beta2, eps,
                       self.adam_step, _stream())
        self.pack()


class Workspace:
    """Activation and gradient buffers of a network of `nlayer` layers for one
    grid shape: h[0 .. nlayer-1] BF16 16-channel activations (the inputs of
    the layers), out FP32, two BF16 gradient buffers."""

    def __init__(self, shape, nlayer=NLAYER):
        import torch
        self.shape = tuple(int(s) for s in shape)
        npts = int(np.prod(self.shape))
        self.h = [torch.zeros((npts, 16), dtype=torch.bfloat16, device="cuda") for _ in range(nlayer)]
        self.out = torch.zeros(npts, dtype=torch.float32, device="cuda")
        self.g = [torch.zeros((npts, 16), dtype=torch.bfloat16, device="cuda") for _ in range(2)]
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")


def features(net, grid, u, u_prev, m, sub, scale, x, stream, noise=0.0, seed=0):
    """The network's input features for grid states u, u_prev and model m;
    `sub` holds the model descriptors (slots of the grid's layout one after
    another) that a network with nsub > 0 reads."""
    if net.nsub:
        fd.fd_cnn_features_sub(grid, u, u_prev, m, sub, net.nsub, scale, net.vref, x, stream, noise=noise, seed=seed)
    else:
        fd.fd_cnn_features(grid, u, u_prev, m, scale, net.vref, x, stream, noise=noise, seed=seed)


def descriptor_slots(grid, sub):
    """Model descriptors [k, *shape] (numpy) copied into slots of the grid's
    padded layout, one after another."""
    import torch
    sub = np.asarray(sub, dtype=np.float32)
    out = torch.zeros((sub.shape[0],) + tuple(grid.padded_shape), dtype=torch.float32, device="cuda")
    out[..., : sub.shape[-1]].copy_(torch.from_numpy(sub))
    return out


def network_forward(net, ws, stream=None, tensor_memory=None):
    """ws.h[0] (features) -> ws.out (FP32, one channel), on the tcgen05
    kernel (tensor_memory True, the default TENSOR_MEMORY) or the mma.sync
    one (False); the two agree to FP32 rounding."""
    st = stream or _stream()
    tensor_memory = TENSOR_MEMORY if tensor_memory is None else tensor_memory
    for li in range(net.nlayer):
        last = li == net.nlayer - 1
        y = ws.out if last else ws.h[li + 1]
        if tensor_memory:
            fd.fd_cnn_conv3d_tc(ws.shape, ws.h[li], net.frag_tc[li], None, net.channels[li + 1], 0 if last else 1, None,
                                y, 1 if last else 0, net.tc_status, st)
        else:
            fd.fd_cnn_conv3d(ws.shape, ws.h[li], net.frag[li], None, net.channels[li + 1], 0 if last else 1, None, y,
                             1 if last else 0, st)


def network_backward(net, ws, stream=None, tensor_memory=None):
    """Accumulate net.grads from dL/dout in ws.g[0] (BF16, channel 0) through
    the activations of the last network_forward."""
    st = stream or _stream()
    tensor_memory = TENSOR_MEMORY if tensor_memory is None else tensor_memory
    cur = 0
    for li in range(net.nlayer - 1, -1, -1):
        cin, cout = net.channels[li], net.channels[li + 1]
        fd.fd_cnn_conv3d_wgrad(ws.shape, ws.h[li], ws.g[cur], cin, cout, net.grad(li), net.gb_dummy, st)
        if li > 0:
            # dL/dh_l = conv(g, flipped W_l) * (h_l > 0): h_l = relu(z_l)
            if tensor_memory:
                fd.fd_cnn_conv3d_tc(ws.shape, ws.g[cur], net.frag_tc_t[li], None, cin, 0, ws.h[li], ws.g[1 - cur], 0,
                                    net.tc_status, st)
            else:
                fd.fd_cnn_conv3d(ws.shape, ws.g[cur], net.frag_t[li], None, cin, 0, ws.h[li], ws.g[1 - cur], 0, st)
            cur = 1 - cur


class ClosureOperator:
    """The coarse operator of a closure_config with the network's correction
    after every step; receivers are recorded like a plain run's."""

    def __init__(self, cfg, net, flags=0):
        import torch
        self.torch = torch
        c = cfg["coarse"]
        self.net = net
        self.shape = c["shape"]
        self.dt = c["dt"]
        self.nt = c["nt"]
        self.grid = fd.Grid(c["shape"], c["spacing"], cfg["origin"])
        self.u = fd.TimeData("u", self.grid)
        self.m = fd.DenseData("m", self.grid)
        self.eta = fd.DenseData("eta", self.grid)
        self.m.data.copy_(torch.from_numpy(c["m"]))
        self.eta.data.copy_(torch.from_numpy(c["eta"]))
        self.src = fd.PointData("src", self.grid, c["src_coords"], self.nt)
        self.src.data[:, : self.src.npoint].copy_(torch.from_numpy(c["src_trace"]))
        self.rec = fd.PointData("rec", self.grid, cfg["rec_coords"], self.nt)
        self.op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, c["space_order"], self.u, self.m, self.eta, src=self.src,
                              rec=self.rec, flags=flags)
        self.sub = descriptor_slots(self.grid, c["sub"][: net.nsub]) if net.nsub else None
        self.ws = Workspace(self.shape, net.nlayer)

    def run(self, nt=None, learned=True):
        """From rest: nt steps (default: the config's), each the coarse update
        plus, when `learned`, the network's correction."""
        nt = self.nt if nt is None else int(nt)
        for s in self.u.slots:
            s.zero_()
        st = _stream()
        g = self.grid.handle
        for n in range(nt):
            if learned:
                features(self.net, g, self.u.slots[n % 2], self.u.slots[(n + 1) % 2], self.m.slots[0], self.sub, 1.0,
                         self.ws.h[0], st)
                network_forward(self.net, self.ws, st)
            self.op.apply(n, 1, self.dt)
            if learned:
                fd.fd_cnn_add_correction(g, self.u.slots[(n + 1) % 2], self.ws.out, self.net.rho, st)
        return self.rec.data[:nt, : self.rec.npoint]


class FineReference:
    """The fine operator of a closure_config (the plain fine-grid run)."""

    def __init__(self, cfg, flags=0, receivers=True):
        import torch
        f = cfg["fine"]
        self.torch = torch
        self.cfg = cfg
        self.shape = f["shape"]
        self.dt = f["dt"]
        self.nt = f["nt"]
        self.grid = fd.Grid(f["shape"], f["spacing"], cfg["origin"])
        self.u = fd.TimeData("u", self.grid)
        self.m = fd.DenseData("m", self.grid)
        self.eta = fd.DenseData("eta", self.grid)
        self.m.data.copy_(torch.from_numpy(f["m"]))
        self.eta.data.copy_(torch.from_numpy(f["eta"]))
        self.src = fd.PointData("src", self.grid, f["src_coords"], self.nt)
        self.src.data[:, : self.src.npoint].copy_(torch.from_numpy(f["src_trace"]))
        self.rec = fd.PointData("rec", self.grid, cfg["rec_coords"], self.nt) if receivers else None
        self.op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, f["space_order"], self.u, self.m, self.eta, src=self.src,
                              rec=self.rec, flags=flags)

    def run(self, nt=None):
        nt = self.nt if nt is None else int(nt)
        for s in self.u.slots:
            s.zero_()
        self.op.apply(0, nt, self.dt)
        return None if self.rec is None else self.rec.data[:nt: 2, : self.rec.npoint]


class Dataset:
    """Training samples of the closure: for coarse steps n of fine runs, the
    restricted fine states R u_f^{n-1}, R u_f^n, R u_f^{n+1}, the coarse step
    S_c(R u_f^n, R u_f^{n-1}) ('base'), the coarse model m and its
    descriptors, and the sample's feature scale s = RMS(R u_f^n)."""

    def __init__(self, cases, steps):
        import torch
        steps = [int(n) for n in steps]
        if steps[0] < 1 or any(b - a < 2 for a, b in zip(steps, steps[1:])):
            raise ValueError("sample steps must start at >= 1 and be at least 2 apart")
        self.torch = torch
        c0 = cases[0]["coarse"]
        self.shape = c0["shape"]
        self.cgrid = fd.Grid(c0["shape"], c0["spacing"], cases[0]["origin"])
        ps = self.cgrid.padded_shape
        ns = len(cases) * len(steps)
        self.states = torch.zeros((ns, 4) + ps, dtype=torch.float32, device="cuda")  # prev, cur, next, base
        self.models = torch.zeros((len(cases),) + ps, dtype=torch.float32, device="cuda")
        self.subs = torch.zeros((len(cases), MAX_SUB) + ps, dtype=torch.float32, device="cuda")
        self.model_of = np.zeros(ns, dtype=np.int64)
        sumsq = torch.zeros(ns, dtype=torch.float32, device="cuda")
        st = _stream()
        k = 0
        for mi, cfg in enumerate(cases):
            cs = cfg["coarse"]
            self.models[mi, ..., : self.shape[2]].copy_(torch.from_numpy(cs["m"]))
            self.subs[mi, ..., : self.shape[2]].copy_(torch.from_numpy(cs["sub"][:MAX_SUB]))
            fine = FineReference(cfg, receivers=False)
            cm = fd.DenseData("m", self.cgrid)
            ce = fd.DenseData("eta", self.cgrid)
            cm.data.copy_(torch.from_numpy(cs["m"]))
            ce.data.copy_(torch.from_numpy(cs["eta"]))
            cu = fd.TimeData("u", self.cgrid)
            csrc = fd.PointData("src", self.cgrid, cs["src_coords"], cs["nt"])
            csrc.data[:, : csrc.npoint].copy_(torch.from_numpy(cs["src_trace"]))
            cop = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, cs["space_order"], cu, cm, ce, src=csrc)
            for s in fine.u.slots:
                s.zero_()
            done = 0
            for n in steps:
                # fine times 2n-2, 2n, 2n+2 -> prev, cur, next
                for j, tf in enumerate((2 * n - 2, 2 * n, 2 * n + 2)):
                    if tf > done:
                        fine.op.apply(done, tf - done, fine.dt)
                        done = tf
                    fd.fd_cnn_restrict(fine.grid.handle, fine.u.slots[tf % 2], self.cgrid.handle,
                                       self.states[k, j], 2, sumsq[k:k + 1] if j == 1 else None, st)
                fd.fd_operator_step(cop.handle, n, cs["dt"], self.states[k, 1].data_ptr(),
                                    self.states[k, 0].data_ptr(), self.states[k, 3].data_ptr())
                self.model_of[k] = mi
                k += 1
        npts = float(np.prod(self.shape))
        self.scale = np.sqrt(np.maximum(sumsq.cpu().numpy().astype(np.float64) / npts, 1e-30))
        self.n = ns

    def residual_ratio(self):
        """rho^2 = mean over samples of mean((next - base)/s)^2: the RMS of the
        residual relative to the wavefield's."""
        torch = self.torch
        ws_pred = torch.zeros(int(np.prod(self.shape)), dtype=torch.float32, device="cuda")
        gy = torch.zeros((ws_pred.numel(), 16), dtype=torch.bfloat16, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        st = _stream()
        for k in range(self.n):
            fd.fd_cnn_mse_grad(self.cgrid.handle, ws_pred, self.states[k, 2], self.states[k, 3], self.scale[k], gy,
                               loss, st)
        return math.sqrt(float(loss.item()) / self.n)


def train(net, data, iters, batch=4, lr=2e-3, seed=0, log_every=0, lr_final=None, noise=0.0):
    """Adam on the mean-squared one-step residual error; returns the loss
    history: (iteration, mean loss per sample over the iterations since the
    previous entry) every `log_every` iterations and at the last.

    noise > 0 perturbs the input states by noise * s (s the sample's RMS) with
    unit-variance uniform deviates while the target stays the clean residual,
    so that the correction does not react to grid-scale content the clean
    samples never show (which a rollout otherwise amplifies)."""
    torch = net.torch
    ws = Workspace(data.shape, net.nlayer)
    g = np.random.default_rng(seed)
    st = _stream()
    hist = []
    lr_final = lr if lr_final is None else lr_final
    ws.loss.zero_()
    since = 0
    for it in range(iters):
        net.grads.zero_()
        since += 1
        for k in g.integers(0, data.n, size=batch):
            s = float(data.scale[k])
            mi = data.model_of[k]
            features(net, data.cgrid.handle, data.states[k, 1], data.states[k, 0], data.models[mi], data.subs[mi], s,
                     ws.h[0], st, noise=noise * s, seed=int(g.integers(0, 2 ** 63)))
            network_forward(net, ws, st)
            fd.fd_cnn_mse_grad(data.cgrid.handle, ws.out, data.states[k, 2], data.states[k, 3], s * net.rho, ws.g[0],
                               ws.loss, st)
            network_backward(net, ws, st)
        # cosine decay from lr to lr_final
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * it / max(iters - 1, 1)))
        net.adam(a)
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, float(ws.loss.item()) / (batch * since)))
            ws.loss.zero_()
            since = 0
    return hist


def train_default(count=128, n_coarse=64, nt=600, iters=800, seed=0, log_every=0, nsub=0, sponge=8):
    """The closure as trained for the evaluation workload: a dataset of
    `count` layered-model runs (workloads.closure_training_set), rho from the
    dataset, 800 Adam iterations of batch 4 with a cosine learning rate from
    2e-3 to 5e-5 (longer training lowered the one-step loss but not the
    rollout error); nsub model descriptors as extra inputs.  Returns (net,
    dataset, loss history)."""
    from . import workloads as wl
    cfgs, steps = wl.closure_training_set(count, n_coarse, nt, sponge=sponge)
    data = Dataset(cfgs, steps)
    net = ClosureNet(seed=seed, rho=data.residual_ratio(), nsub=nsub)
    hist = train(net, data, iters, batch=4, lr=2e-3, lr_final=5e-5, seed=seed, log_every=log_every)
    return net, data, hist


def trace_error(traces, reference):
    """Relative L2 error of receiver traces against the fine-grid traces."""
    a = np.asarray(traces, dtype=np.float64)
    b = np.asarray(reference, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
