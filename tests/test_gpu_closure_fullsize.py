"""The closure network at the size the learned benchmark runs it: 128^3 coarse
points, 6 -> 16 -> 16 -> 16 -> 1 channels, 3^3 kernels, BF16 weights and
activations, FP32 accumulation, on the tcgen05 convolution (the closure's
default).  Its outputs are checked at sampled points against the oracle's
network (oracle/cnn.py), which computes each one from the 9^3 block of
inputs around it.

Why a block suffices: four 3^3 layers give each output a receptive field of
9^3 inputs.  For the block clipped to the grid, at the grid's faces the
block's zero padding is the network's own; at the block's interior faces
the zero padding reaches only values that the centre does not depend on.
(Layer l at offset k from the centre needs layer l - 1 at offsets up to
k + 1, so the centre needs layer 1 only within 3 of it, computed from
inputs within 4.)

Tolerance: as for the network on small grids (test_gpu_closure.py).  The
oracle stores the three hidden activations in BF16, as the device does, so
only the FP32 accumulation order differs, and the sampled outputs match to
1e-3 in relative L2.
"""
import numpy as np
import pytest

from oracle import cnn

pytestmark = pytest.mark.gpu

N = 128
R = 4  # receptive-field radius of the 4-layer network


def _samples(seed):
    g = np.random.default_rng(seed)
    pts = [tuple(int(v) for v in g.integers(0, N, size=3)) for _ in range(160)]
    # faces, edges and corners, where the padding matters
    for a in (0, 1, R - 1, R, N - R - 1, N - 1):
        pts.append((a, int(g.integers(0, N)), int(g.integers(0, N))))
        pts.append((int(g.integers(0, N)), a, int(g.integers(0, N))))
        pts.append((int(g.integers(0, N)), int(g.integers(0, N)), a))
    pts += [(i, j, k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]
    # around the kernel's tile seams (4-row tile columns of 128 points, 4-plane steps)
    pts += [(63, 3, 64), (64, 4, 0), (31, 7, 127), (32, 8, 1), (100, 63, 5), (101, 64, 126)]
    return pts


def test_network_full_size_sampled_against_oracle():
    torch = pytest.importorskip("torch")
    from paper_1707_03776_gb300 import closure
    shape = (N, N, N)
    net = closure.ClosureNet(seed=11, rho=1.0)
    cin = net.channels[0]
    ws = closure.Workspace(shape)
    g = np.random.default_rng(12)
    x = np.zeros(shape + (16,), dtype=np.float32)
    x[..., :cin] = g.standard_normal(shape + (cin,)).astype(np.float32)
    xr = cnn.bf16_round(x)
    ws.h[0].copy_(torch.from_numpy(xr.reshape(-1, 16)).to(torch.bfloat16).cuda())
    closure.network_forward(net, ws)
    net.check()
    out = ws.out.cpu().numpy().reshape(shape)

    params = [(cnn.bf16_round(w).astype(np.float64), np.zeros(w.shape[2])) for w in net.weights()]
    x64 = xr[..., :cin].astype(np.float64)
    got, want = [], []
    for p in _samples(13):
        lo = [max(c - R, 0) for c in p]
        hi = [min(c + R + 1, N) for c in p]
        block = x64[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        acts, _ = cnn.network_forward(block, params, store=cnn.bf16_round)
        want.append(acts[-1][p[0] - lo[0], p[1] - lo[1], p[2] - lo[2], 0])
        got.append(out[p])
    got = np.array(got, dtype=np.float64)
    want = np.array(want)
    assert np.all(np.isfinite(got)) and np.linalg.norm(want) > 0
    print("%d sampled outputs: relative L2 %.3e, max abs %.3e of max %.3e" % (
        len(got), np.linalg.norm(got - want) / np.linalg.norm(want), np.abs(got - want).max(), np.abs(want).max()))
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), np.linalg.norm(got - want) / np.linalg.norm(want)
