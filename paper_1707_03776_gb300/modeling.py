"""Forward modelling with host inputs and outputs: the paper's `forward()`
(Seismic Inversion Example) as one call a user makes.

AcousticModel keeps every device buffer resident between calls; `forward`
copies the host model (m, eta), the source wavelet and coordinates-derived
tables are set up once, runs the whole time loop through the C ABI and copies
the receiver traces back.  Host tensors should be pinned for asynchronous
copies.
"""
import time

import numpy as np

from . import fd


class AcousticModel:
    def __init__(self, shape, spacing, origin, space_order, src_coords, rec_coords, nt, flags=0):
        import torch
        self.torch = torch
        self.shape = tuple(int(s) for s in shape)
        self.nt = int(nt)
        self.space_order = int(space_order)
        self.grid = fd.Grid(self.shape, spacing, origin)
        self.u = fd.TimeData("u", self.grid)
        self.m = fd.DenseData("m", self.grid)
        self.eta = fd.DenseData("eta", self.grid)
        self.m.data.fill_(1.0)
        self.src = fd.PointData("src", self.grid, src_coords, self.nt)
        self.rec = fd.PointData("rec", self.grid, rec_coords, self.nt)
        self.op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, self.space_order, self.u, self.m, self.eta,
                              src=self.src, rec=self.rec, flags=flags)
        self.rec_host = torch.empty((self.nt, self.rec.npoint), dtype=torch.float32, pin_memory=True)

    def h2d_bytes(self):
        n = int(np.prod(self.shape))
        return 2 * 4 * n + 4 * self.nt * self.src.npoint

    def d2h_bytes(self):
        return 4 * self.nt * self.rec.npoint

    def load(self, m, eta, src_trace):
        """Copy host inputs to the device (non-blocking from pinned memory)."""
        torch = self.torch
        as_t = lambda a: a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))  # noqa
        self.m.data.copy_(as_t(m).reshape(self.shape), non_blocking=True)
        self.eta.data.copy_(as_t(eta).reshape(self.shape), non_blocking=True)
        self.src.data[:, : self.src.npoint].copy_(as_t(src_trace).reshape(self.nt, -1), non_blocking=True)
        # rebinding recomputes min(m) for the stability check and marks the
        # coefficient fields stale
        self.op.bind("m", self.m)
        self.op.bind("eta", self.eta)

    def autotune(self, dt, nsteps=20):
        """Pick the fastest tiling on this model's data (leaves u zeroed);
        the trial runs take at most the model's nt steps."""
        nsteps = max(1, min(int(nsteps), self.nt))
        for s in self.u.slots:
            s.zero_()
        best = fd.fd_operator_autotune(self.op.handle, 0, nsteps, dt)
        for s in self.u.slots:
            s.zero_()
        self.op.sync()
        return best

    def run(self, dt):
        """One forward run from rest on device-resident inputs."""
        for s in self.u.slots:
            s.zero_()
        self.op.apply(0, self.nt, dt)

    def forward(self, m, eta, src_trace, dt, timings=None):
        """Host m, eta, src trace in -> host receiver traces [nt, nrec] out.

        With a dict `timings`, the host-side phases of the call are added to
        it in seconds (no extra synchronisation): "load" (the copies in and
        the min(m) check, which waits for them), "launch" (enqueueing the
        time loop and the copy back) and "wait" (until the traces are on the
        host)."""
        t0 = time.perf_counter()
        self.load(m, eta, src_trace)
        t1 = time.perf_counter()
        self.run(dt)
        self.rec_host.copy_(self.rec.data[:, : self.rec.npoint], non_blocking=True)
        t2 = time.perf_counter()
        self.torch.cuda.current_stream().synchronize()
        self.op.sync()
        if timings is not None:
            t3 = time.perf_counter()
            timings["load"] = t1 - t0
            timings["launch"] = t2 - t1
            timings["wait"] = t3 - t2
        return self.rec_host
