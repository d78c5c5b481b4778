"""Parity of the CUDA diffusion path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from fdrun import rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def run_diffusion(u0, spacing, so, a, dt, nt, flags=0):
    import torch
    grid = fd.Grid(u0.shape, spacing)
    u = fd.TimeData("u", grid)
    u.at(0).copy_(torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)))
    op = fd.Operator(fd.FD_DIFFUSION_EULER, so, u, a=a, flags=flags)
    op.apply(0, nt, dt)
    op.sync()
    return u.at(nt).cpu().numpy(), op


def test_ring_workload_full_run():
    """The 256^2 ring, 500 steps: the whole run against the oracle."""
    cfg = wl.diffusion_ring()
    got, op = run_diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"])
    ref = oracle.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"])
    assert rel_l2(got, ref) <= 1e-5
    assert got.min() >= -1e-6 and got.max() <= 1.0 + 1e-6


def test_one_step_parity_orders():
    for so, shape in [(2, (37, 75)), (4, (64, 129)), (8, (19, 23, 71)), (16, (40, 41))]:
        h = tuple(1.0 / (n + 1) for n in shape)
        u0 = wl.random_field(shape, so, smooth=1)
        dt = 0.05 * min(h) ** 2
        got, _ = run_diffusion(u0, h, so, 0.7, dt, 1)
        ref = oracle.diffusion(u0.astype(np.float64), h, so, 0.7, dt, 1)
        assert rel_l2(got, ref) <= 1e-6, (so, shape)


def test_unstable_dt_rejected():
    cfg = wl.diffusion_ring(n=64)
    with pytest.raises(fd.FDError) as e:
        run_diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], 2.6 * cfg["dt"] / 0.2 * 0.2 * 5, 1)
    assert e.value.status == fd.FD_ERR_UNSTABLE
