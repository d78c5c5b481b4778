"""Test helpers: run the CUDA path through the C ABI (paper_1707_03776_gb300.fd)
on numpy inputs and bring results back as numpy arrays."""
import numpy as np

from paper_1707_03776_gb300 import fd


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


class AcousticRun:
    """A GPU acoustic operator over numpy inputs."""

    def __init__(self, shape, spacing, origin, space_order, m, eta=None, src_coords=None, src_trace=None,
                 rec_coords=None, n_total=1, flags=0):
        import torch
        self.torch = torch
        self.grid = fd.Grid(shape, spacing, origin)
        self.u = fd.TimeData("u", self.grid)
        self.m = fd.DenseData("m", self.grid)
        self.m.data.copy_(torch.from_numpy(np.ascontiguousarray(m, dtype=np.float32)))
        self.eta = None
        if eta is not None:
            self.eta = fd.DenseData("eta", self.grid)
            self.eta.data.copy_(torch.from_numpy(np.ascontiguousarray(eta, dtype=np.float32)))
        self.src = self.rec = None
        if src_coords is not None:
            self.src = fd.PointData("src", self.grid, src_coords, n_total)
            self.src.data[:, : self.src.npoint].copy_(
                torch.from_numpy(np.ascontiguousarray(src_trace, dtype=np.float32).reshape(n_total, -1)))
        if rec_coords is not None:
            self.rec = fd.PointData("rec", self.grid, rec_coords, n_total)
        self.op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, space_order, self.u, self.m, self.eta,
                              src=self.src, rec=self.rec, flags=flags)

    def set_state(self, u_cur, u_prev, t0=0):
        torch = self.torch
        self.u.at(t0).copy_(torch.from_numpy(np.ascontiguousarray(u_cur, dtype=np.float32)))
        self.u.at(t0 + 1).copy_(torch.from_numpy(np.ascontiguousarray(u_prev, dtype=np.float32)))

    def run(self, t0, nt, dt):
        self.op.apply(t0, nt, dt)
        self.op.sync()

    def state(self, n):
        """(u^n, u^{n-1}) after a forward run that ended at time n."""
        return self.u.at(n).cpu().numpy().copy(), self.u.at(n + 1).cpu().numpy().copy()

    def rec_trace(self):
        return self.rec.data[:, : self.rec.npoint].cpu().numpy().copy()
