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


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS], ids=["cluster", "plain"])
def test_ring_workload_full_run(flags):
    """The 256^2 ring, 500 steps: the whole run against the oracle."""
    cfg = wl.diffusion_ring()
    got, op = run_diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"], flags=flags)
    ref = oracle.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"])
    assert rel_l2(got, ref) <= 1e-5
    assert got.min() >= -1e-6 and got.max() <= 1.0 + 1e-6


@pytest.mark.parametrize("flags", [0, fd.FD_FLAG_PLAIN_KERNELS], ids=["cluster", "plain"])
def test_one_step_parity_orders(flags):
    for so, shape in [(2, (37, 75)), (4, (64, 129)), (8, (19, 23, 71)), (16, (140, 41)), (6, (300, 333))]:
        h = tuple(1.0 / (n + 1) for n in shape)
        u0 = wl.random_field(shape, so, smooth=1)
        dt = 0.05 * min(h) ** 2
        got, _ = run_diffusion(u0, h, so, 0.7, dt, 1, flags=flags)
        ref = oracle.diffusion(u0.astype(np.float64), h, so, 0.7, dt, 1)
        assert rel_l2(got, ref) <= 1e-6, (so, shape)


@pytest.mark.parametrize("nt", [2, 7, 40])
def test_multi_step_and_slots(nt):
    """Several steps in one cluster launch: both slots hold the last two
    states, as with per-step launches."""
    shape = (90, 77)
    h = (1.0 / 91, 1.0 / 78)
    u0 = wl.random_field(shape, 3, smooth=2)
    dt = 0.2 * min(h) ** 2 / 0.5
    import torch
    outs = []
    for flags in (0, fd.FD_FLAG_PLAIN_KERNELS):
        grid = fd.Grid(shape, h)
        u = fd.TimeData("u", grid)
        u.at(3).copy_(torch.from_numpy(u0))
        op = fd.Operator(fd.FD_DIFFUSION_EULER, 4, u, a=0.5, flags=flags)
        op.apply(3, nt, dt)
        op.sync()
        outs.append((u.at(3 + nt).cpu().numpy(), u.at(3 + nt - 1).cpu().numpy()))
    ref = oracle.diffusion(u0.astype(np.float64), h, 4, 0.5, dt, nt)
    ref_prev = oracle.diffusion(u0.astype(np.float64), h, 4, 0.5, dt, nt - 1)
    for last, prev in outs:
        assert rel_l2(last, ref) <= 1e-5
        assert rel_l2(prev, ref_prev) <= 1e-5


def test_unstable_dt_rejected():
    cfg = wl.diffusion_ring(n=64)
    with pytest.raises(fd.FDError) as e:
        run_diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], 2.6 * cfg["dt"] / 0.2 * 0.2 * 5, 1)
    assert e.value.status == fd.FD_ERR_UNSTABLE
