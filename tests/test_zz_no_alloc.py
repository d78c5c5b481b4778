"""fd_interpolate_noalloc: receiver interpolation for callers that cannot
allocate device memory when they record (memory fully reserved by another
allocator's pool, a fixed budget set at start-up, a loop that must not risk
the device-wide synchronisation of cudaMalloc/cudaFree).  Its table lives in a
fixed static device array instead.

Checked through the C ABI, on two calls in a row with different points and
fields (so that the second call cannot pass on the first call's table):
  * against the interpolation the operator performs (rec[0] = R u^0 of
    fd_operator_apply), and against the FP64 oracle's trilinear
    interpolation of the same FP32 field, both within 1e-6 relative L2;
  * that after the set-up call (no points) the calls change neither the
    device's free memory (cudaMemGetInfo) nor torch's reserved memory.
This file is collected last on purpose.
"""
import gc

import numpy as np
import pytest

import oracle
from fdrun import rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-6
CASES = [((36, 41, 70), 3000, 1), ((23, 50, 33), 777, 2), ((60, 47), 1500, 3)]


def operator_interpolation(grid, field_np, coords):
    """rec[0] of a one-step acoustic run from u^0 = field: the existing path."""
    import torch
    u = fd.TimeData("u", grid)
    u.at(0).copy_(torch.from_numpy(field_np))
    m = fd.DenseData("m", grid)
    m.data.fill_(1.0 / 2000.0 ** 2)
    rec = fd.PointData("rec", grid, coords, 1)
    op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 4, u, m, rec=rec)
    op.apply(0, 1, 1e-3)
    op.sync()
    return rec.data[0, : rec.npoint].cpu().numpy(), u, (op, rec, m)


def _prepare():
    """Inputs, the operator's and the oracle's interpolation for every case;
    every allocation is done here, before the calls under test."""
    import torch
    out = []
    for shape, npoint, seed in CASES:
        h = tuple(10.0 + a for a in range(len(shape)))
        origin = tuple(-5.0 * a for a in range(len(shape)))
        grid = fd.Grid(shape, h, origin)
        field = wl.random_field(shape, seed)
        coords = wl.random_points(shape, h, origin, npoint, seed)
        ref_op, u, keep = operator_interpolation(grid, field, coords)
        ref_or = oracle.interpolate_from_f32(field, h, origin, coords)
        dst = torch.full((npoint,), float("nan"), dtype=torch.float32, device="cuda")
        out.append((grid, coords, u, dst, ref_op, ref_or, keep))
    # nothing made before the calls under test may be freed during them (a
    # free returns memory to the device and would move the free count)
    gc.collect()
    torch.cuda.synchronize()
    return out


def test_noalloc_matches_operator_and_oracle_twice_without_allocating():
    import torch
    stream = torch.cuda.current_stream()
    # set-up on this device: loads the static table and the kernel
    fd.fd_interpolate_noalloc(None, None, 0, 0, stream.cuda_stream)
    cases = _prepare()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for rep in range(2):
        for grid, coords, u, dst, ref_op, ref_or, _ in cases:
            dst.fill_(float("nan"))
            fd.fd_interpolate_noalloc(grid.handle, coords, u.slots[0].data_ptr(), dst.data_ptr(),
                                      stream.cuda_stream)
            stream.synchronize()
            got = dst.cpu().numpy()
            assert np.isfinite(got).all()
            assert rel_l2(got, ref_op) <= TOL, (rep, coords.shape, "operator")
            assert rel_l2(got, ref_or) <= TOL, (rep, coords.shape, "oracle")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "device free memory moved by %d bytes" % (free0 - free1)
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_oversized_requests():
    import torch
    grid = fd.Grid((8, 9, 10), (1.0, 1.0, 1.0))
    out = torch.zeros(4, device="cuda")
    field = torch.zeros((8, 9, 16), device="cuda")
    coords = np.zeros((fd.FD_NOALLOC_MAX_POINTS + 1, 3))
    with pytest.raises(fd.FDError) as e:
        fd.fd_interpolate_noalloc(grid.handle, coords, field.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == fd.FD_ERR_INVALID_ARG
    assert str(fd.FD_NOALLOC_MAX_POINTS) in str(e.value)
    with pytest.raises(fd.FDError) as e:
        fd.fd_interpolate_noalloc(grid.handle, np.array([[0.0, 0.0, 9.5]]), field.data_ptr(), out.data_ptr(), 0)
    assert e.value.status == fd.FD_ERR_OUT_OF_DOMAIN
