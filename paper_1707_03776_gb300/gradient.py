"""Adjoint-state gradient of the acoustic forward operator with respect to m,
with checkpointing, behind a torch.autograd.Function.

Forward: the operator of the Seismic Inversion Example run from rest; every
`checkpoint_every` steps the two wavefield levels are copied aside -- or,
when the whole history fits in device memory (256^3 x 1500 steps is 100 GB
of the GPU's 280 GB), every state is kept and nothing is recomputed.
Backward: the paper's adjoint operator (the same update run backward in time
with the receiver residual injected, FD_FLAG_REVERSE) sweeps the checkpoint
segments from last to first; inside each segment the forward states are
recomputed from its checkpoint with out-of-place steps (fd_operator_step) into
a segment buffer, and the imaging condition
    dJ/dm += -(1/dt^2) mu^n (u^n - 2u^{n-1} + u^{n-2})
is accumulated in the same pass as every adjoint step where the tiled sweep
injects the residual itself (fd_operator_apply_imaging: fused into the
sweep).  Otherwise up to four adjoint steps run first, out of place into a
ring of six adjoint states, and one pass images them all
(fd_imaging_accumulate_steps), reading each forward state and the gradient
once for the four steps.  Either way the gradient is the same bit for bit.

Every step of the path runs in libfdgb's kernels; torch provides the device
memory (fields, checkpoints, the segment buffer) and the autograd plumbing.
"""
import numpy as np

from . import fd


class Shot:
    """One seismic experiment: source positions and wavelets, receiver
    positions, on a grid."""

    def __init__(self, src_coords, src_trace, rec_coords):
        self.src_coords = np.ascontiguousarray(src_coords, dtype=np.float64)
        self.src_trace = np.ascontiguousarray(src_trace, dtype=np.float32)
        self.rec_coords = np.ascontiguousarray(rec_coords, dtype=np.float64)


class Propagator:
    """Device-resident forward and adjoint operators for one grid and shot."""

    def __init__(self, shape, spacing, origin, space_order, shot, nt, dt, checkpoint_every=None, flags=0):
        """checkpoint_every: k > 0 keeps two states every k steps and
        recomputes the segments in the backward sweep; 0 keeps the whole
        forward history in device memory (no recomputation); None picks 0
        when the history takes at most half the free device memory, else 50."""
        import torch
        self.torch = torch
        self.shape = tuple(int(s) for s in shape)
        self.nt = int(nt)
        self.dt = float(dt)
        self.grid = fd.Grid(self.shape, spacing, origin)
        slot_bytes = 4 * int(np.prod(self.grid.padded_shape))
        if checkpoint_every is None:
            free, _ = torch.cuda.mem_get_info()
            checkpoint_every = 0 if (self.nt + 2) * slot_bytes <= free // 2 else 50
        self.k = int(checkpoint_every)
        self.m = fd.DenseData("m", self.grid)
        self.eta = fd.DenseData("eta", self.grid)
        self.m.data.fill_(1.0)
        self.u = fd.TimeData("u", self.grid)
        self.src = fd.PointData("src", self.grid, shot.src_coords, self.nt)
        self.src.data[:, : self.src.npoint].copy_(torch.from_numpy(shot.src_trace.reshape(self.nt, -1)))
        self.rec = fd.PointData("rec", self.grid, shot.rec_coords, self.nt)
        # forward with receivers; recomputation without them
        self.fwd = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, space_order, self.u, self.m, self.eta, src=self.src,
                               rec=self.rec, flags=flags)
        self.re = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, space_order, self.u, self.m, self.eta, src=self.src,
                              flags=flags)
        # adjoint: residual injected at the receiver positions, backward in time
        self.mu = fd.TimeData("mu", self.grid)
        self.res = fd.PointData("res", self.grid, shot.rec_coords, self.nt)
        self.adj = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, space_order, self.mu, self.m, self.eta, src=self.res,
                               flags=flags | fd.FD_FLAG_REVERSE)
        ps = self.grid.padded_shape
        if self.k > 0:
            nseg = (self.nt + self.k - 1) // self.k
            # checkpoint j: the states of times jk-1 and jk-2 (zero for j = 0)
            self.ckpt = torch.zeros((nseg, 2) + ps, dtype=torch.float32, device="cuda")
            # segment buffer: states of times jk-2 .. (j+1)k-1
            self.seg = torch.zeros((self.k + 2,) + ps, dtype=torch.float32, device="cuda")
        else:
            # the whole history: hist[i] holds the state of time i-1 (-1 .. nt)
            self.hist = torch.zeros((self.nt + 2,) + ps, dtype=torch.float32, device="cuda")
        self.grad = fd.DenseData("grad", self.grid)
        self.stream = torch.cuda.current_stream().cuda_stream
        # adjoint states of times t in ring[t % 6] (steps out of place, imaged four at a time)
        self.mu_ring = torch.zeros((6,) + ps, dtype=torch.float32, device="cuda")

    def set_damping(self, eta):
        """Damping eta (held fixed by the gradient)."""
        torch = self.torch
        t = eta if isinstance(eta, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(eta, dtype=np.float32))
        self.eta.data.copy_(t.reshape(self.shape))
        for op in (self.fwd, self.re, self.adj):
            op.bind("eta", self.eta)

    def set_model(self, m, eta=None):
        torch = self.torch
        self.m.data.copy_(m.reshape(self.shape))
        if eta is not None:
            self.eta.data.copy_(eta.reshape(self.shape))
        for op in (self.fwd, self.re, self.adj):
            op.bind("m", self.m)
            op.bind("eta", self.eta)

    def forward(self):
        """Forward run from rest with checkpoints (or the whole history);
        returns the device traces."""
        if self.k == 0:
            hist = self.hist
            hist[0].zero_()
            hist[1].zero_()
            for n in range(self.nt):
                fd.fd_operator_step(self.fwd.handle, n, self.dt, hist[n + 1].data_ptr(), hist[n].data_ptr(),
                                    hist[n + 2].data_ptr())
            return self.rec.data[:, : self.rec.npoint]
        for s in self.u.slots:
            s.zero_()
        self.ckpt[0].zero_()
        k = self.k
        done = 0
        for j in range(1, self.ckpt.shape[0]):
            # run up to time jk-1, then keep u^{jk-1} (slot (jk-1)%2) and
            # u^{jk-2} (the other slot)
            t = j * k - 1
            self.fwd.apply(done, t - done, self.dt)
            done = t
            self.ckpt[j, 0].copy_(self.u.slots[t % 2])
            self.ckpt[j, 1].copy_(self.u.slots[(t + 1) % 2])
        self.fwd.apply(done, self.nt - done, self.dt)
        return self.rec.data[:, : self.rec.npoint]

    def backward(self, residual):
        """Adjoint run with `residual` [nt, nrec] injected; returns dJ/dm as an
        interior view (grid shape) of the library's gradient buffer."""
        torch = self.torch
        self.res.data[:, : self.res.npoint].copy_(residual)
        for s in self.mu.slots:
            s.zero_()
        self.mu_ring.zero_()
        self.grad.slots[0].zero_()
        scale = -1.0 / (self.dt * self.dt)
        if self.k == 0:
            hist = self.hist
            self._adjoint_steps(self.nt - 1, 0, lambda t: hist[t + 1].data_ptr(), scale)
            return self.grad.data
        k = self.k
        seg = self.seg
        for j in range(self.ckpt.shape[0] - 1, -1, -1):
            n_lo = j * k
            n_hi = min((j + 1) * k, self.nt)
            # seg[i] holds the state of time n_lo - 2 + i
            seg[1].copy_(self.ckpt[j, 0])
            seg[0].copy_(self.ckpt[j, 1])
            for t in range(n_lo - 1, n_hi - 1):
                i = t - (n_lo - 2)
                if t < 0:
                    # u^0 from rest: only the source term of step -1 is absent
                    seg[i + 1].zero_()
                    continue
                fd.fd_operator_step(self.re.handle, t, self.dt, seg[i].data_ptr(), seg[i - 1].data_ptr(),
                                    seg[i + 1].data_ptr())
            self._adjoint_steps(n_hi - 1, n_lo, lambda t, lo=n_lo: seg[t - (lo - 2)].data_ptr(), scale)
        return self.grad.data

    def _adjoint_steps(self, n_top, n_bot, state, scale):
        """Adjoint steps n_top .. n_bot (backward) with the imaging condition;
        state(t) is the device pointer of the forward state of time t, for
        t >= n_bot - 2."""
        gp = self.grad.slots[0].data_ptr()
        if fd.fd_operator_sources_fused(self.adj.handle):
            # the sweep images the state it writes, one step at a time
            for n in range(n_top, n_bot - 1, -1):
                if n >= 1:
                    fd.fd_operator_apply_imaging(self.adj.handle, n, self.dt, scale, state(n), state(n - 1),
                                                 state(n - 2), gp)
                else:
                    self.adj.apply(n, 1, self.dt)
            return
        # up to four steps out of place into the ring, then one pass images
        # them; the adjoint state of time 0 images nothing and is not computed
        ring = self.mu_ring
        lo = max(n_bot, 1)
        n = n_top
        while n >= lo:
            k = min(4, n - lo + 1)
            for t in range(n, n - k, -1):
                fd.fd_operator_step(self.adj.handle, t, self.dt, ring[(t + 1) % 6].data_ptr(),
                                    ring[(t + 2) % 6].data_ptr(), ring[t % 6].data_ptr())
            fd.fd_imaging_accumulate_steps(self.grid.handle, scale, [ring[(n - j) % 6].data_ptr() for j in range(k)],
                                           [state(n - i) for i in range(k + 2)], gp, self.stream)
            n -= k


def _autograd_function():
    import torch

    class AcousticModelling(torch.autograd.Function):
        """rec = F(m): forward modelling; backward = adjoint-state gradient."""

        @staticmethod
        def forward(ctx, m, prop):
            prop.set_model(m)
            rec = prop.forward().clone()
            ctx.prop = prop
            return rec

        @staticmethod
        def backward(ctx, grad_rec):
            g = ctx.prop.backward(grad_rec.contiguous()).clone()
            return g, None

    return AcousticModelling


_FN = None


def modelling(m, prop):
    """Differentiable forward modelling: receiver traces of the shot of `prop`
    for square slowness m (a CUDA tensor of the grid's shape)."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(m, prop)
