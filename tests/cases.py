"""Small runnable cases of each kernel family, for profiling one kernel at a
time (python tests/cases.py <case> [options]).

Each case builds its inputs from the seeded workloads, runs a few warm-up
launches, then `--reps` launches of the kernel of interest, synchronises and
exits 0.  Sizes default to inputs larger than L2 (129 MB) with a few GB on
the device at most.

  acoustic   the tiled grid update (512^3 SO8 by default)
  pair       the same run with two time steps per sweep (the two-step kernel)
  batch      the batched-shots persistent kernel (8 windows of the 512^3 model)
  gradient   forward, checkpoint recomputation, adjoint and imaging of one
             shot (256^3 SO8, 100 steps, checkpoints every 10 steps)
  diffusion  the 2D diffusion cluster kernel (256^2 ring, 500 steps per run)
  conv       the closure network's forward convolutions (160^3 activations)
  conv_tc    the same on the tcgen05 kernel
  wgrad      the closure network's weight-gradient kernel (96^3)
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _sync():
    import torch
    torch.cuda.synchronize()


def case_acoustic(args):
    import torch
    from paper_1707_03776_gb300 import fd, workloads as wl
    from paper_1707_03776_gb300.modeling import AcousticModel
    cfg = wl.acoustic_config(n=args.n, space_order=args.so, nt=args.nt)
    model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], args.so, cfg["src_coords"],
                          cfg["rec_coords"], args.nt)
    model.load(torch.from_numpy(cfg["m"]), torch.from_numpy(cfg["eta"]), torch.from_numpy(cfg["src_trace"]))
    if args.tiling:
        rows, stages = (int(x) for x in args.tiling.split(","))
        fd.fd_operator_set_tiling(model.op.handle, rows, stages)
    model.run(cfg["dt"])
    model.op.sync()
    _sync()


def case_pair(args):
    import torch
    from paper_1707_03776_gb300 import fd, workloads as wl
    from paper_1707_03776_gb300.modeling import AcousticModel
    cfg = wl.acoustic_config(n=args.n, space_order=args.so, nt=args.nt)
    model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], args.so, cfg["src_coords"],
                          cfg["rec_coords"], args.nt)
    model.load(torch.from_numpy(cfg["m"]), torch.from_numpy(cfg["eta"]), torch.from_numpy(cfg["src_trace"]))
    fd.fd_operator_set_time_block(model.op.handle, 2)
    model.run(cfg["dt"])
    model.op.sync()
    _sync()


def case_batch(args):
    import torch
    from paper_1707_03776_gb300 import fd, workloads as wl
    cfg = wl.batched_config(nshots=args.shots, nt=args.nt)
    keep = []
    ops = []
    for i in range(args.shots):
        shape, m, eta, src, rec = wl.window_shot(cfg, i)
        grid = fd.Grid(shape, cfg["spacing"])
        u = fd.TimeData("u", grid)
        md, ed = fd.DenseData("m", grid), fd.DenseData("eta", grid)
        md.data.copy_(torch.from_numpy(m))
        ed.data.copy_(torch.from_numpy(eta))
        sp = fd.PointData("src", grid, src, args.nt)
        sp.data[:, :1].copy_(torch.from_numpy(cfg["wavelet"]))
        rp = fd.PointData("rec", grid, rec, args.nt)
        op = fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, u, md, ed, src=sp, rec=rp)
        keep.append((grid, u, md, ed, sp, rp))
        ops.append(op)
    batch = fd.Batch(ops, rows=args.rows, stages=args.stages)
    batch.apply(0, args.nt, cfg["dt"])
    batch.sync()
    _sync()


def case_gradient(args):
    import torch
    from paper_1707_03776_gb300 import workloads as wl
    from paper_1707_03776_gb300.gradient import Propagator, Shot, modelling
    cfg = wl.gradient_config(n=args.n, nt=args.nt)
    prop = Propagator(cfg["shape"], cfg["spacing"], cfg["origin"], 8,
                      Shot(cfg["shots"][0], cfg["wavelet"], cfg["rec_coords"]), args.nt, cfg["dt"],
                      checkpoint_every=min(10, args.nt))
    prop.set_damping(cfg["eta"])
    prop.set_model(torch.from_numpy(cfg["m_true"]).cuda())
    d_obs = prop.forward().clone()
    m = torch.from_numpy(cfg["m0"]).cuda().requires_grad_(True)
    rec = modelling(m, prop)
    (0.5 * ((rec - d_obs) ** 2).sum()).backward()
    _sync()


def case_diffusion(args):
    import torch
    from paper_1707_03776_gb300 import fd, workloads as wl
    cfg = wl.diffusion_ring()
    grid = fd.Grid(cfg["shape"], cfg["spacing"], cfg["origin"])
    u = fd.TimeData("u", grid)
    op = fd.Operator(fd.FD_DIFFUSION_EULER, 2, u, a=cfg["a"])
    u0 = torch.from_numpy(cfg["u0"]).cuda()
    for _ in range(args.reps):
        u.at(0).copy_(u0)
        op.apply(0, cfg["nt"], cfg["dt"])
    op.sync()
    _sync()


def case_conv(args):
    import torch
    from paper_1707_03776_gb300 import closure, fd
    net = closure.ClosureNet(seed=0, rho=1e-3)
    shape = (args.n,) * 3
    ws = closure.Workspace(shape)
    g = torch.Generator(device="cuda").manual_seed(0)
    ws.h[0].copy_(torch.randn(ws.h[0].shape, generator=g, device="cuda").to(torch.bfloat16))
    ws.h[0][:, 6:].zero_()
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(args.reps):
        closure.network_forward(net, ws, st, tensor_memory=False)
    _sync()


def case_conv_tc(args):
    import torch
    from paper_1707_03776_gb300 import closure
    net = closure.ClosureNet(seed=0, rho=1e-3)
    shape = (args.n,) * 3
    ws = closure.Workspace(shape)
    g = torch.Generator(device="cuda").manual_seed(0)
    ws.h[0].copy_(torch.randn(ws.h[0].shape, generator=g, device="cuda").to(torch.bfloat16))
    ws.h[0][:, 6:].zero_()
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(args.reps):
        closure.network_forward(net, ws, st, tensor_memory=True)
    _sync()


def case_wgrad(args):
    import torch
    from paper_1707_03776_gb300 import closure, fd
    shape = (args.n,) * 3
    npts = int(np.prod(shape))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn((npts, 16), generator=g, device="cuda").to(torch.bfloat16)
    gy = torch.randn((npts, 16), generator=g, device="cuda").to(torch.bfloat16)
    gw = torch.zeros((27, 16, 16), dtype=torch.float32, device="cuda")
    gb = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(args.reps):
        fd.fd_cnn_conv3d_wgrad(shape, x, gy, 16, 16, gw, gb, st)
    _sync()


CASES = {"acoustic": case_acoustic, "pair": case_pair, "batch": case_batch, "gradient": case_gradient, "diffusion": case_diffusion,
         "conv": case_conv, "conv_tc": case_conv_tc, "wgrad": case_wgrad}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("case", choices=sorted(CASES))
    p.add_argument("--n", type=int, default=None, help="grid points per axis")
    p.add_argument("--so", type=int, default=8)
    p.add_argument("--nt", type=int, default=None, help="time steps")
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--shots", type=int, default=8)
    p.add_argument("--rows", type=int, default=16)
    p.add_argument("--stages", type=int, default=2)
    p.add_argument("--tiling", default="", help="rows,stages of the tiled kernel")
    args = p.parse_args(argv)
    defaults = {"acoustic": (512, 10), "pair": (512, 10), "batch": (None, 10), "gradient": (256, 100), "diffusion": (256, 500),
                "conv": (160, None), "conv_tc": (160, None), "wgrad": (96, None)}
    n, nt = defaults[args.case]
    args.n = args.n or n
    args.nt = args.nt or nt
    t0 = time.perf_counter()
    CASES[args.case](args)
    print("case %s done in %.2f s" % (args.case, time.perf_counter() - t0))


if __name__ == "__main__":
    main()
