"""The batched-shots workload at its configured size, in the configuration the
batched benchmark times: 64 SO8 shots on windows of 160^3 to 320^3 of the
512^3 random smooth model, 800 steps, the tiling chosen by fd_batch_autotune,
one launch per step, eager and as a replayed CUDA graph.

* Every shot's receiver traces and final field equal those of the same
  operator run alone, bit for bit: each grid point gets the same arithmetic
  in either kernel.
* The smallest window's traces match the FP32 oracle run of that window to
  1e-4 in relative L2 (the full-run trace gate).
"""
import numpy as np
import pytest

import oracle
from fdrun import rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4


def test_batched_workload_full_size():
    import torch
    cfg = wl.batched_config()
    nt, dt = cfg["nt"], cfg["dt"]
    shots = []
    for i in range(len(cfg["windows"])):
        shape, m, eta, src, rec = wl.window_shot(cfg, i)
        grid = fd.Grid(shape, cfg["spacing"])
        u = fd.TimeData("u", grid)
        md = fd.DenseData("m", grid)
        ed = fd.DenseData("eta", grid)
        md.data.copy_(torch.from_numpy(m))
        ed.data.copy_(torch.from_numpy(eta))
        sp = fd.PointData("src", grid, src, nt)
        sp.data[:, :1].copy_(torch.from_numpy(cfg["wavelet"]))
        rp = fd.PointData("rec", grid, rec, nt)
        op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u, md, ed, src=sp, rec=rp)
        shots.append(dict(u=u, rec=rp, op=op, shape=shape, args=(shape, m, eta, src, rec)))

    def reset():
        for s in shots:
            for t in s["u"].slots:
                t.zero_()

    def results():
        return [(s["rec"].data[:, : s["rec"].npoint].clone(), s["u"].at(nt).clone()) for s in shots]

    # each operator alone
    reset()
    for s in shots:
        s["op"].apply(0, nt, dt)
        s["op"].sync()
    alone = results()

    batch = fd.Batch([s["op"] for s in shots])
    reset()
    batch.autotune(0, 20, dt)
    for mode in ("eager", "graph"):
        reset()
        if mode == "eager":
            batch.apply(0, nt, dt)
        else:
            batch.capture(0, nt, dt)
            batch.replay()
        batch.sync()
        for i, ((tr, u), (tr_a, u_a)) in enumerate(zip(results(), alone)):
            assert torch.equal(tr, tr_a), (mode, i)
            assert torch.equal(u, u_a), (mode, i)

    k = int(np.argmin([np.prod(s["shape"]) for s in shots]))
    shape, m, eta, src, rec = shots[k]["args"]
    _, _, orec = oracle.acoustic_forward(shape, cfg["spacing"], (0.0, 0.0, 0.0), 8, m, eta, dt, nt,
                                         src_coords=src, src_trace=cfg["wavelet"], rec_coords=rec, precision="f32")
    err = rel_l2(alone[k][0].cpu().numpy(), orec)
    print("window %s: traces against the FP32 oracle, relative L2 %.3e" % (shape, err))
    assert err <= TRACE_TOL
