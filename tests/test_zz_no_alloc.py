"""fd_interpolate_noalloc: receiver interpolation for callers that cannot
allocate device memory (its table lives in a fixed static device array).

Checked through the C ABI against the interpolation the operator performs
(rec[0] = R u^0 of fd_operator_apply), on two calls in a row with different
points and fields, so that the second call cannot pass on the first call's
table.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from fdrun import rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-6


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
    return rec.data[0, : rec.npoint].cpu().numpy(), u


def test_noalloc_matches_operator_interpolation_twice():
    import torch
    cases = [((36, 41, 70), 3000, 1), ((23, 50, 33), 777, 2), ((60, 47), 1500, 3)]
    for shape, npoint, seed in cases:
        h = tuple(10.0 + a for a in range(len(shape)))
        origin = tuple(-5.0 * a for a in range(len(shape)))
        grid = fd.Grid(shape, h, origin)
        field = wl.random_field(shape, seed)
        coords = wl.random_points(shape, h, origin, npoint, seed)
        ref, u = operator_interpolation(grid, field, coords)
        out = torch.full((npoint,), float("nan"), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        fd.fd_interpolate_noalloc(grid.handle, coords, u.slots[0].data_ptr(), out.data_ptr(),
                                  stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, (shape, npoint)


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
