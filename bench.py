#!/usr/bin/env python
"""Benchmark: 3D isotropic acoustic forward modelling, 512^3, SO8, 1000 steps.

One bench step is one whole forward run of the hot path on synthetic inputs
shaped like the paper's 512^3 benchmark: coefficient preparation
(c = dt^2/m, d = dt*eta/m), then 1000 time steps of receiver interpolation
(101 x 101 receivers), the SO8 leapfrog update with sponge damping, and
Ricker source injection.  Inputs (fields of 0.5 GB each) are resident in HBM
and larger than L2, so no L2 flush is needed between steps.

Printed (rank 0): one JSON line with the throughput in GPts/s (interior points
x time steps / second), the roofline of the grid-update kernel (HBM bound, 20
algorithmic bytes per point per step), the CPU oracle timed on this host's
cores on a bounded sample, an end-to-end figure through the host-buffer API,
kernel launches in the timed region and the SM clocks seen meanwhile.

`--impl reference` times the CPU oracle instead (the only reference this
paper has: there is no reference code), on bounded samples of the same
workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D acoustic SO8 GPts/s & %HBM roofline; learned/batched vs plain at equal error"
BYTES_PER_POINT = 20  # read u^n, u^{n-1}, c, d; write u^{n+1} (FP32)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--so", type=int, default=8)
    p.add_argument("--nt", type=int, default=1000)
    p.add_argument("--cpu-steps", type=int, default=3, help="time steps in the CPU-oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-rows", action="store_true", help="skip the secondary rows")
    p.add_argument("--rows", default="space_orders,diffusion,convection,laplace,gradient,batched,learned,two_step",
                   help="secondary rows to run (comma-separated)")
    p.add_argument("--plain", action="store_true", help="plain kernels instead of the tiled ones")
    p.add_argument("--tiling", default="", help="rows,stages of the tiled kernel (default: autotuned)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value, world):
    """The largest of every rank's value (all ranks receive it): the job's
    time is its slowest replica's.  Uses the default process group when
    world > 1 (a CUDA tensor under NCCL, a CPU one under gloo)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_step, steps, world, seconds):
    """GPts/s of the whole job: every rank runs its own replica (weak
    scaling), so the points of all ranks over the slowest rank's time."""
    return points_per_step * steps * world / seconds / 1e9


def workload_name(n, so, nt):
    return "acoustic3d_%d^3_so%d_nt%d_1src_101x101rec_sponge40" % (n, so, nt)


def config_dict(args):
    return {"workload": workload_name(args.n, args.so, args.nt), "grid": [args.n] * 3, "space_order": args.so,
            "time_order": 2, "nt": args.nt, "h_m": 10.0, "cfl": 0.4, "velocity": "1500/2500 m/s two-layer",
            "sponge_cells": 40, "sources": 1, "receivers": 101 * 101,
            "l2": "inputs larger than L2 (0.5 GB per field), no flush",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------

def oracle_sample(cfg, so, steps, precision="f32"):
    """Time `steps` oracle time steps of the forward run on the full grid."""
    import numpy as np
    import oracle
    n_total = cfg["nt"]
    t = time.perf_counter()
    oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["m"], cfg["eta"], cfg["dt"],
                            steps, src_coords=cfg["src_coords"], src_trace=cfg["src_trace"],
                            rec_coords=cfg["rec_coords"], n_total=n_total, precision=precision)
    dt = time.perf_counter() - t
    pts = float(np.prod(cfg["shape"])) * steps
    return pts / dt / 1e9, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1707_03776_gb300 import workloads as wl
    oracle._lib()
    cfg = wl.acoustic_config(n=args.n, space_order=args.so, nt=args.nt)
    steps_per = max(1, args.cpu_steps)
    for _ in range(args.warmup):
        oracle_sample(cfg, args.so, steps_per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(cfg, args.so, steps_per)
    el = time.perf_counter() - t0
    value = args.n ** 3 * steps_per * args.steps / el / 1e9
    sample = "%d of %d time steps of the forward run per bench step, full %d^3 grid, FP32 loop nest" % (
        steps_per, args.nt, args.n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GPts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_dict(args),
            "cpu_baseline": {"value": value, "unit": "GPts/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GPts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "note": "the paper ships no code; the reference arm is the plain CPU oracle (OpenMP loop nest)"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    def __init__(self, index):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(REASONS, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def measured_peak_bf16():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except Exception:
        return 1900.0, "fallback"


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    """First 16 hex digits of the SHA-256 of the grid-update kernel's source:
    k_tma.cu followed by the column sweep it instantiates, k_sweep.cuh."""
    h = hashlib.sha256()
    for f in ("k_tma.cu", "k_sweep.cuh"):
        with open(os.path.join(ROOT, "paper_1707_03776_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(so):
    """DRAM bytes per launch of the grid-update kernel from the committed ncu
    summary, if it was taken on the kernel source as it is now."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = kernel_source_sha()
        entry = rec.get("so%d" % so)
        if entry and entry.get("source_sha") == sha:
            return float(entry["bytes_per_launch_512"])
    except Exception:
        pass
    return None


def bench_diffusion(steps=5, warmup=3):
    """The 2D diffusion row (256^2 ring, 500 explicit Euler steps), timed
    with CUDA events: the grid is L2/shared-memory resident, so it is reported
    as time per step, not against the HBM roofline."""
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    cfg = wl.diffusion_ring()
    grid = fd.Grid(cfg["shape"], cfg["spacing"], cfg["origin"])
    u = fd.TimeData("u", grid)
    u0 = torch.from_numpy(cfg["u0"]).cuda()
    op = fd.Operator(fd.FD_DIFFUSION_EULER, 2, u, a=cfg["a"])
    stream = torch.cuda.current_stream()

    def run():
        u.at(0).copy_(u0)
        op.apply(0, cfg["nt"], cfg["dt"])

    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    n0 = op.launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    op.sync()
    ms = e0.elapsed_time(e1) / steps
    pts = float(cfg["shape"][0] * cfg["shape"][1]) * cfg["nt"]
    k, ctas = fd.fd_operator_get_time_block(op.handle)
    import oracle
    cpu = _cpu_oracle(lambda: oracle.diffusion(cfg["u0"], cfg["spacing"], 2, cfg["a"], cfg["dt"], cfg["nt"],
                                               precision="f32"), pts, "GPts/s", "the whole 500-step run, FP32")
    return {"workload": "diffusion2d_256^2_ring_so2_nt500", "value": pts / (ms * 1e-3) / 1e9, "unit": "GPts/s",
            "ms_per_run": ms, "us_per_time_step": 1e3 * ms / cfg["nt"],
            "launches_per_run": (op.launches - n0) / steps, "cluster_ctas": ctas, "steps_per_exchange": k,
            "bound": "latency (grid held in one cluster's shared memory)", "cpu_oracle": cpu}


def _cpu_oracle(fn, pts, unit, sample):
    """Time one bounded oracle call on the host cores (a reported baseline
    beside each row, not a target)."""
    import oracle
    oracle._lib()
    t = time.perf_counter()
    fn()
    el = time.perf_counter() - t
    return {"value": pts / el / 1e9, "unit": unit, "cores": oracle.num_threads(), "kind": "oracle",
            "s": el, "sample": sample}


def _time_runs(fn, reps, warmup=3):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_convection(reps=20):
    """The Linear Convection example (81^2, c = 1, 100 upwind steps): one
    cluster launch per run; against the plain per-step kernels."""
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    cfg = wl.convection_config()
    grid = fd.Grid(cfg["shape"], cfg["spacing"])
    u = fd.TimeData("u", grid)
    u0 = torch.from_numpy(cfg["u0"]).cuda()
    out = {}
    for name, flags in (("cluster", 0), ("plain", fd.FD_FLAG_PLAIN_KERNELS)):
        op = fd.Operator(fd.FD_CONVECTION_UPWIND, 1, u, a=cfg["c"], flags=flags)

        def run():
            u.at(0).copy_(u0)
            op.apply(0, cfg["nt"], cfg["dt"])

        out[name] = _time_runs(run, reps)
        if name == "cluster":
            k, ctas = fd.fd_operator_get_time_block(op.handle)
        op.sync()
    pts = float(cfg["shape"][0] * cfg["shape"][1]) * cfg["nt"]
    import oracle
    cpu = _cpu_oracle(lambda: oracle.convection(cfg["u0"], cfg["spacing"], cfg["c"], cfg["dt"], cfg["nt"],
                                                precision="f32"), pts, "GPts/s", "the whole 100-step run, FP32")
    return {"cpu_oracle": cpu, "workload": "convection2d_81^2_c1_nt100", "value": pts / (out["cluster"] * 1e-3) / 1e9,
            "unit": "GPts/s", "ms_per_run": out["cluster"], "us_per_time_step": 1e3 * out["cluster"] / cfg["nt"],
            "plain_ms_per_run": out["plain"], "speedup_vs_plain": out["plain"] / out["cluster"],
            "cluster_ctas": ctas, "steps_per_exchange": k}


def bench_laplace(reps=5):
    """The Laplace example (31^2 on [0,2]x[0,1], Dirichlet rows, Neumann
    columns) to the L1 criterion 1e-4: the whole convergence loop in one
    cluster launch that decides on the device; against per-sweep launches
    with the sum read back every sweep."""
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    cfg = wl.laplace_config()
    grid = fd.Grid(cfg["shape"], cfg["spacing"])
    u = fd.TimeData("u", grid)
    p0 = torch.from_numpy(cfg["p0"]).cuda()
    out = {}
    for name, flags in (("cluster", 0), ("plain", fd.FD_FLAG_PLAIN_KERNELS)):
        op = fd.Operator(fd.FD_LAPLACE_JACOBI, 2, u, flags=flags)
        res = []

        def run():
            u.at(0).copy_(p0)
            res.append(op.converge(0, 1000000, cfg["tol"]))

        run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            run()
        out[name] = ((time.perf_counter() - t0) / reps * 1e3, res[-1])
    it = out["cluster"][1][0]
    import oracle
    npts = float(cfg["shape"][0] * cfg["shape"][1]) * it
    cpu = _cpu_oracle(lambda: oracle.laplace(cfg["p0"], cfg["spacing"], cfg["tol"], 1000000, precision="f32"),
                      npts, "GPts/s (sweeps x points / s)", "the whole convergence loop, FP32")
    cpu["ms"] = cpu["s"] * 1e3
    return {"cpu_oracle": cpu, "workload": "laplace2d_31^2_tol1e-4", "unit": "ms to convergence", "value": out["cluster"][0],
            "sweeps": it, "r_last": out["cluster"][1][1], "us_per_sweep": 1e3 * out["cluster"][0] / it,
            "plain_ms": out["plain"][0], "plain_sweeps": out["plain"][1][0],
            "speedup_vs_plain": out["plain"][0] / out["cluster"][0]}


def bench_gradient(n=256, nt=1500, k=50, shots=8):
    """The adjoint/gradient row: dJ/dm summed over the 8 shots of the 256^3 SO8
    workload (1500 steps, 65x65 receivers each), with checkpoints every 50
    steps (the forward states of each segment recomputed in the backward
    sweep, the imaging fused into the adjoint sweep).  Beside it, per shot:
    the same with the whole forward history kept in HBM (100 GB, nothing
    recomputed) and with the plain kernels, at equal result (relative
    differences given)."""
    import numpy as np
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    from paper_1707_03776_gb300.gradient import Propagator, Shot, modelling
    cfg = wl.gradient_config(n=n, nt=nt, nshots=shots)
    m_true = torch.from_numpy(cfg["m_true"]).cuda()
    m0 = torch.from_numpy(cfg["m0"]).cuda()

    def propagator(shot, kk, flags=0):
        prop = Propagator(cfg["shape"], cfg["spacing"], cfg["origin"], 8, Shot(shot, cfg["wavelet"], cfg["rec_coords"]),
                          nt, cfg["dt"], checkpoint_every=kk, flags=flags)
        prop.set_damping(cfg["eta"])
        # observed data: the true model through the same forward operator
        prop.set_model(m_true)
        return prop, prop.forward().clone()

    def gradient(props, reps=2):
        """min over reps of the time of dJ/dm over the propagators' shots."""
        times = []
        for _ in range(reps):
            m = m0.clone().requires_grad_(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            total = 0.0
            for prop, d_obs in props:
                rec = modelling(m, prop)
                loss = 0.5 * ((rec - d_obs) ** 2).sum()
                loss.backward()
                total += float(loss.item())
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        return min(times), m.grad.detach().double(), total

    # headline: all shots, checkpoints every k steps
    props = [propagator(shot, k) for shot in cfg["shots"]]
    fused = all(fd.fd_operator_sources_fused(p.adj.handle) for p, _ in props)
    launches0 = sum(p.adj.launches + p.re.launches + p.fwd.launches for p, _ in props)
    s_all, g_all, loss_all = gradient(props, reps=2)
    launches = (sum(p.adj.launches + p.re.launches + p.fwd.launches for p, _ in props) - launches0) // 2
    del props
    torch.cuda.empty_cache()
    # per-shot comparisons on the first shot
    side = {}
    grads = {}
    for name, flags, kk in (("checkpointed", 0, k), ("whole_history", 0, 0), ("plain", fd.FD_FLAG_PLAIN_KERNELS, k)):
        pr = [propagator(cfg["shots"][0], kk, flags)]
        t, g, _ = gradient(pr, reps=2 if name != "plain" else 1)
        side[name] = t
        grads[name] = g
        del pr
        torch.cuda.empty_cache()
    g_c = grads["checkpointed"]
    rel_hist = float((grads["whole_history"] - g_c).norm() / g_c.norm())
    rel_plain = float((grads["plain"] - g_c).norm() / g_c.norm())
    pts = float(n) ** 3 * nt
    import oracle
    sc = wl.gradient_config(n=64, nt=100, nrec_side=17, sponge=10)
    nrec = sc["rec_coords"].shape[0]
    cpu = _cpu_oracle(lambda: oracle.acoustic_gradient(
        sc["shape"], sc["spacing"], sc["origin"], 8, sc["m0"].astype(np.float64), sc["eta"].astype(np.float64),
        sc["dt"], 100, sc["shots"][0], sc["wavelet"][:100], sc["rec_coords"], np.zeros((100, nrec))),
        64.0 ** 3 * 100, "GPts/s (grid points x steps / s of forward+adjoint+imaging)",
        "64^3 SO8, 100 steps, 17x17 receivers, FP64 loop nest keeping the whole history")
    return {"workload": "gradient3d_%d^3_so8_nt%d_%dshots_65x65rec" % (n, nt, shots),
            "shots": shots, "checkpoint_every": k,
            "value": shots * pts / s_all / 1e9,
            "unit": "GPts/s (grid points x steps of the modelled shots per second of forward+adjoint+imaging)",
            "s_gradient_all_shots": s_all, "s_per_shot": s_all / shots, "loss": loss_all,
            "launches_per_gradient": launches,
            "imaging": ("fused into the adjoint sweep with the residual injection (fd_operator_apply_imaging)"
                        if fused else "up to four adjoint steps out of place, then one pass imaging them "
                        "(fd_imaging_accumulate_steps; the sweep does not stage the adjoint's sources)"),
            "adjoint_sources_fused": fused,
            "recomputed_steps_per_shot": nt,
            "per_shot": {"checkpointed_s": side["checkpointed"],
                         "whole_history_s": side["whole_history"],
                         "whole_history_GB": (nt + 2) * 4 * n ** 3 / 1e9,
                         "plain_kernels_s": side["plain"],
                         "speedup_vs_plain": side["plain"] / side["checkpointed"],
                         "grad_rel_diff_whole_history_vs_checkpointed": rel_hist,
                         "grad_rel_diff_plain_vs_checkpointed": rel_plain},
            "cpu_oracle": cpu}


def bench_batched(nshots=64, nt=800, plain_shots=8):
    """The batched-shots row: 64 SO8 shots on windows of 160^3-320^3 of a
    512^3 smooth random model, 800 steps; one launch per step for all shots
    (eager and as a replayed CUDA graph, tile height autotuned over a short
    run) against the same shots run one after another with the single-shot
    tiled operator and with the plain kernels (the latter on `plain_shots`
    shots, scaled), at equal receiver traces."""
    import numpy as np
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    cfg = wl.batched_config(nshots=nshots, nt=nt)
    dt = cfg["dt"]
    shots = []
    for i in range(nshots):
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
        shots.append(dict(grid=grid, u=u, m=md, eta=ed, src=sp, rec=rp, op=op, shape=shape))
    pts = float(sum(np.prod(s["shape"]) for s in shots)) * nt

    def reset():
        for s in shots:
            for t in s["u"].slots:
                t.zero_()

    def timed(fn):
        reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    # sequential single-shot runs (each operator's own planner tiling)
    t_seq = timed(lambda: [s["op"].apply(0, nt, dt) for s in shots])
    traces_seq = [s["rec"].data[:, :s["rec"].npoint].clone() for s in shots[:plain_shots]]
    # sequential plain-kernel runs on a subset
    plain_ops = [fd.Operator(fd.FD_ACOUSTIC_LEAPFROG, 8, s["u"], s["m"], s["eta"], src=s["src"], rec=s["rec"],
                             flags=fd.FD_FLAG_PLAIN_KERNELS) for s in shots[:plain_shots]]
    t_plain_sub = timed(lambda: [op.apply(0, nt, dt) for op in plain_ops])
    traces_plain = [s["rec"].data[:, :s["rec"].npoint].clone() for s in shots[:plain_shots]]
    pts_sub = float(sum(np.prod(s["shape"]) for s in shots[:plain_shots])) * nt
    del plain_ops
    # the library's autotuner picks the batch's tile height and depth on a
    # short run of its own data
    batch = fd.Batch([s["op"] for s in shots])
    reset()
    tuned = batch.autotune(0, 20, dt)
    info = batch.info()
    batch.apply(0, 5, dt)
    batch.sync()
    t_batch = timed(lambda: batch.apply(0, nt, dt))
    batch.capture(0, nt, dt)
    t_graph = timed(lambda: batch.replay())
    batch.sync()
    traces_b = [s["rec"].data[:, :s["rec"].npoint] for s in shots[:plain_shots]]
    err = max(float((a - b).norm() / b.norm()) for a, b in zip(traces_b, traces_plain))
    err_seq = max(float((a - b).norm() / b.norm()) for a, b in zip(traces_b, traces_seq))
    import oracle
    shape0, m0_, eta0, src0, rec0 = wl.window_shot(cfg, 0)
    cpu = _cpu_oracle(lambda: oracle.acoustic_forward(shape0, cfg["spacing"], (0.0, 0.0, 0.0), 8, m0_, eta0, dt, 3,
                                                      src_coords=src0, src_trace=cfg["wavelet"], rec_coords=rec0,
                                                      n_total=nt, precision="f32"),
                      float(np.prod(shape0)) * 3, "GPts/s", "3 steps of the first window %s, FP32" % (shape0,))
    return {"cpu_oracle": cpu, "workload": "batched_%dshots_windows160-320_of_512^3_so8_nt%d" % (nshots, nt),
            "value": pts / t_graph / 1e9, "unit": "GPts/s (sum of window points x steps / s)",
            "s_batch_graph": t_graph, "s_batch_eager": t_batch, "s_sequential_tiled": t_seq,
            "s_sequential_plain_est": t_plain_sub * pts / pts_sub,
            "speedup_vs_sequential_plain": (t_plain_sub * pts / pts_sub) / t_graph,
            "speedup_vs_sequential_tiled": t_seq / t_graph,
            "trace_rel_diff_vs_plain": err, "trace_rel_diff_vs_sequential_tiled": err_seq,
            "tiling": {"rows_per_tile": info[0], "prefetch_planes": info[1], "ctas": info[2],
                       "source": "fd_batch_autotune", "autotuned_ms_per_step": tuned[2]},
            "launches_per_step": 1, "window_points": pts / nt}


def bench_space_orders(n=512, nt=100, reps=3, orders=(2, 4, 8, 12, 16)):
    """The 512^3 forward workload (source, 10 201 receivers, sponge) at every
    space order the method covers: time per step of the whole run, the grid
    update's own time from CUDA events on its launches and its fraction of the
    measured HBM bandwidth at 20 bytes per point, and one step of the FP32
    oracle on the host cores beside it."""
    import torch
    import oracle
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    from paper_1707_03776_gb300.modeling import AcousticModel
    peak, kind = measured_peak_hbm()
    out = {"workload": "acoustic3d_%d^3_nt%d_1src_101x101rec_sponge40" % (n, nt), "peak_kind": kind}
    for so in orders:
        cfg = wl.acoustic_config(n=n, space_order=so, nt=nt)
        model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["src_coords"], cfg["rec_coords"],
                              nt)
        model.load(cfg["m"], cfg["eta"], cfg["src_trace"])
        model.run(cfg["dt"])
        model.op.sync()
        model.op.profile(reps * nt)
        ms = _time_runs(lambda: model.run(cfg["dt"]), reps, warmup=0) / nt
        model.op.sync()
        k_ms, k_n = model.op.profile_read()
        kms = k_ms / k_n if k_n else None
        rows, stages, ctas = fd.fd_operator_get_tiling(model.op.handle)
        v, el = oracle_sample(cfg, so, 1)
        out["SO%d" % so] = {
            "ms_per_step": ms, "GPts_per_s": float(n) ** 3 / (ms * 1e-3) / 1e9, "kernel_ms": kms,
            "roofline_frac": (BYTES_PER_POINT * float(n) ** 3 / (kms * 1e-3) / 1e9 / peak) if kms else None,
            "tiling": {"rows_per_tile": rows, "prefetch_planes": stages, "ctas": ctas},
            "cpu_oracle": {"value": v, "unit": "GPts/s", "cores": oracle.num_threads(), "s": el,
                           "sample": "1 step, FP32"}}
        del model
        torch.cuda.empty_cache()
    return out


def bench_two_step(n=512, so=8, nt=200, reps=3):
    """Temporal blocking of the grid update: the headline forward workload
    (512^3 SO8, source and receivers) run with one and with two time steps
    per sweep on the same operator, bitwise-equal results checked.  The
    two-step sweep's own HBM traffic is 24 bytes per point per launch (u^n,
    u^{n-1}, c, d read; u^{n+1}, u^{n+2} written), so its roofline is
    effective bandwidth = 40 bytes per point per launch / kernel time."""
    import torch
    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    from paper_1707_03776_gb300.modeling import AcousticModel
    cfg = wl.acoustic_config(n=n, space_order=so, nt=nt)
    model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], so, cfg["src_coords"], cfg["rec_coords"], nt)
    model.load(cfg["m"], cfg["eta"], cfg["src_trace"])
    op = model.op
    out, res = {}, {}
    for k in (1, 2):
        fd.fd_operator_set_time_block(op.handle, k)
        kk, ctas = fd.fd_operator_get_time_block(op.handle)

        def run():
            for s in model.u.slots:
                s.zero_()
            op.apply(0, nt, cfg["dt"])

        run()
        op.sync()
        op.profile(reps * nt)
        ms = _time_runs(run, reps, warmup=1) / nt
        op.sync()
        k_ms, k_n = op.profile_read()
        res[k] = [t.clone() for t in model.u.slots]
        out["steps_per_sweep_%d" % k] = {
            "ms_per_time_step": ms, "GPts_per_s": float(n) ** 3 / (ms * 1e-3) / 1e9, "ctas": ctas,
            "sweep_ms_avg": (k_ms / k_n) if k_n else None, "time_steps_per_sweep": kk}
    same = all(torch.equal(a, b) for a, b in zip(res[1], res[2]))
    two = out["steps_per_sweep_2"]
    peak, peak_kind = measured_peak_hbm()
    if two["sweep_ms_avg"]:
        s_ = two["sweep_ms_avg"] * 1e-3
        two["hbm_GBs_own_traffic"] = 24.0 * n ** 3 / s_ / 1e9
        two["effective_GBs"] = 40.0 * n ** 3 / s_ / 1e9
        two["effective_frac_of_measured_hbm"] = two["effective_GBs"] / peak
    return {"workload": workload_name(n, so, nt), "bitwise_equal": bool(same),
            "speedup_two_vs_one": out["steps_per_sweep_1"]["ms_per_time_step"] / two["ms_per_time_step"],
            "peak_kind": peak_kind, **out}


def bench_learned(n=128, nt=2000):
    """The learned-closure row: a coarse 20 m SO4 grid corrected every step
    by the 4-layer BF16 CNN, trained on 128 fine-grid (10 m, SO16) runs of
    seeded layered models, evaluated on an unseen layered model on a 256^3-
    equivalent domain (128^3 coarse, 255^3 fine nodes) for 2000 coarse steps.
    Receiver-trace errors are relative to the plain fine-grid run (the
    reference); the plain coarse grid at SO 4/8/16 shows what the spatial order
    alone buys at 20 m.  Wall times include every launch of the run (the
    network, the coarse update, the correction)."""
    import numpy as np
    import torch
    from paper_1707_03776_gb300 import closure
    from paper_1707_03776_gb300 import workloads as wl

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    (net, data, hist), t_train = timed(lambda: closure.train_default(log_every=200))
    n_samples = data.n
    cfg = wl.closure_config(n, nt, seed=1001, src="surface")
    fine = closure.FineReference(cfg)
    fine.run(20)
    ref, t_fine = timed(lambda: fine.run().cpu().numpy())
    del fine
    plain = {}
    for so in (4, 8, 16):
        c2 = dict(cfg)
        c2["coarse"] = dict(cfg["coarse"], space_order=so)
        op = closure.ClosureOperator(c2, net)
        op.run(20, learned=False)
        tr, t = timed(lambda: op.run(learned=False).cpu().numpy())
        plain["SO%d" % so] = {"trace_rel_err": closure.trace_error(tr, ref), "s": t}
        del op
    op = closure.ClosureOperator(cfg, net)
    op.run(20)
    lr_tr, t_learned = timed(lambda: op.run().cpu().numpy())
    err = closure.trace_error(lr_tr, ref)
    # the same comparison with a 24-cell sponge: with the thin 8-cell sponge
    # the traces are dominated by boundary reverberations, which differ
    # between the grids; the thick sponge leaves the interior propagation
    cfg24 = wl.closure_config(n, nt, seed=1001, src="surface", sponge=24)
    fine24 = closure.FineReference(cfg24)
    ref24 = fine24.run().cpu().numpy()
    del fine24
    op24 = closure.ClosureOperator(cfg24, net)
    thick = {"sponge_cells": 24,
             "trace_rel_err_plain_coarse_SO4": closure.trace_error(op24.run(learned=False).cpu().numpy(), ref24),
             "trace_rel_err_learned": closure.trace_error(op24.run().cpu().numpy(), ref24)}
    del op24
    # a closure that also sees where the coarse model misplaces interfaces
    # (two sub-cell descriptors), trained on 8- and 24-cell sponges alike
    del data
    (net_d, data_d, hist_d), t_train_d = timed(
        lambda: closure.train_default(n_coarse=96, nsub=2, sponge=(8, 24), log_every=200))
    del data_d
    errs_d = {}
    for sp, c, r in ((8, cfg, ref), (24, cfg24, ref24)):
        o = closure.ClosureOperator(c, net_d)
        errs_d["sponge%d" % sp] = closure.trace_error(o.run().cpu().numpy(), r)
        del o
    thick["with_interface_descriptors"] = {
        "nsub": 2, "train_models": "128 at 96^3 coarse, sponges 8 and 24 alternately", "train_s": t_train_d,
        "loss_first_last": [hist_d[0][1], hist_d[-1][1]] if hist_d else None,
        "trace_rel_err_learned_sponge8": errs_d["sponge8"], "trace_rel_err_learned_sponge24": errs_d["sponge24"]}
    net_d.check()
    del net_d
    # the network alone: CUDA events around its launches
    st = torch.cuda.current_stream()
    for _ in range(3):
        closure.network_forward(net, op.ws, st.cuda_stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(st)
    for _ in range(reps):
        closure.network_forward(net, op.ws, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    ms_net = e0.elapsed_time(e1) / reps
    # the same network on the mma.sync kernel (equal to FP32 rounding; for
    # comparison)
    for _ in range(3):
        closure.network_forward(net, op.ws, st.cuda_stream, tensor_memory=False)
    e0.record(st)
    for _ in range(reps):
        closure.network_forward(net, op.ws, st.cuda_stream, tensor_memory=False)
    e1.record(st)
    torch.cuda.synchronize()
    ms_net_mma = e0.elapsed_time(e1) / reps
    pts = float(n) ** 3
    ch = net.channels
    flops = 2.0 * 27 * pts * sum(ch[i] * ch[i + 1] for i in range(len(ch) - 1))
    flops_mma = 2.0 * 27 * pts * 16 * 16 * 4  # issued: channels padded to 16 on both sides of every layer
    peak, kind = measured_peak_bf16()
    achieved = flops / (ms_net * 1e-3) / 1e12
    from oracle import cnn
    wts = [(w.astype(np.float64), np.zeros(w.shape[2])) for w in net.weights()]
    xs = np.random.default_rng(0).standard_normal((32, 32, 32, 6))
    cpu = _cpu_oracle(lambda: cnn.network_forward(xs, wts), 2.0 * 27 * 32 ** 3 * sum(
        ch[i] * ch[i + 1] for i in range(len(ch) - 1)) / 1e3, "TFLOP/s",
        "network forward on 32^3 points, numpy FP64")
    return {"workload": "closure_coarse%d^3_20m_so4_fine%d^3_10m_so16_nt%d_layered" % (n, 2 * n - 1, nt),
            "unit": "s per modelled shot; trace errors relative to the fine grid",
            "trace_rel_err_learned": err, "trace_rel_err_plain_coarse": plain, "thick_sponge_check": thick,
            "s_learned": t_learned, "s_fine_grid": t_fine,
            "learned_vs_fine_time": t_learned / t_fine,
            "train": {"s": t_train, "samples": n_samples, "models": 128, "iters": 800, "rho": net.rho,
                      "loss_first_last": [hist[0][1], hist[-1][1]]},
            "network_ms_per_step": ms_net, "network_share_of_learned_step": ms_net * nt / 1e3 / t_learned,
            "network_ms_per_step_mma_sync": ms_net_mma,
            "cpu_oracle": cpu,
            "roofline": {"bound": "tensor",
                         "kernel": "conv3d on tcgen05 (BF16 operands in shared memory, N <= 48 MMAs over three d1 "
                                   "taps, FP32 accumulators in TMEM)",
                         "achieved": achieved, "achieved_mma_issued": flops_mma / (ms_net * 1e-3) / 1e12,
                         "peak": peak, "peak_kind": kind, "unit": "TFLOP/s", "frac": achieved / peak}}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1707_03776_gb300 import fd
    from paper_1707_03776_gb300 import workloads as wl
    from paper_1707_03776_gb300.modeling import AcousticModel

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    cfg = wl.acoustic_config(n=args.n, space_order=args.so, nt=args.nt)
    flags = fd.FD_FLAG_PLAIN_KERNELS if args.plain else 0
    model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], args.so, cfg["src_coords"],
                          cfg["rec_coords"], args.nt, flags=flags)
    m_h = torch.from_numpy(cfg["m"]).pin_memory()
    eta_h = torch.from_numpy(cfg["eta"]).pin_memory()
    src_h = torch.from_numpy(cfg["src_trace"]).pin_memory()
    model.load(m_h, eta_h, src_h)
    tiling = None
    if not args.plain and args.tiling:
        rows, stages = (int(x) for x in args.tiling.split(","))
        fd.fd_operator_set_tiling(model.op.handle, rows, stages)
        r, s_, ctas = fd.fd_operator_get_tiling(model.op.handle)
        tiling = {"rows_per_tile": r, "prefetch_planes": s_, "ctas": ctas, "source": "--tiling"}
    elif not args.plain:
        rows, stages, ms_tuned = model.autotune(cfg["dt"])
        tiling = {"rows_per_tile": rows, "prefetch_planes": stages, "autotuned_ms_per_step": ms_tuned,
                  "ctas": fd.fd_operator_get_tiling(model.op.handle)[2]}
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    op = model.op

    def step():
        # coefficients are recomputed every step (a2), then the whole time loop
        op.bind("eta", model.eta)
        model.run(cfg["dt"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    op.sync()

    op.profile(args.steps * args.nt)
    launches0 = op.launches
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = op.launches - launches0
    op.sync()
    k_ms, k_n = op.profile_read()
    ms_max = max_over_ranks(ms, world)
    pts = float(args.n) ** 3 * args.nt
    value = whole_job_rate(pts, args.steps, world, ms_max * 1e-3)

    # receivers must hold a finite, non-trivial shot record
    rec = model.rec.data[:, : model.rec.npoint]
    assert torch.isfinite(rec).all().item() and rec.abs().max().item() > 0

    e2e = None
    if not args.no_e2e:
        # each step (one forward call: host model in, traces out) timed on its
        # own; the median of five, because the host-side part of a call (the
        # copies and the launches) varies from call to call: on some hosts a
        # 1 GB copy from pinned memory takes 6 ms in one call and 45 ms in
        # the next
        e_steps = 5
        model.forward(m_h, eta_h, src_h, cfg["dt"])  # warm
        barrier()
        els, phases = [], []
        for _ in range(e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ph = {}
            out = model.forward(m_h, eta_h, src_h, cfg["dt"], timings=ph)
            torch.cuda.synchronize()
            els.append(max_over_ranks(time.perf_counter() - t0, world))
            phases.append({k: round(v * 1e3, 3) for k, v in ph.items()})
        el = sorted(els)[len(els) // 2]
        e2e = {"value": whole_job_rate(pts, 1, world, el), "unit": "GPts/s",
               "h2d_bytes_per_step": model.h2d_bytes(), "d2h_bytes_per_step": model.d2h_bytes(),
               "steps": e_steps, "stat": "median of the steps", "s_per_step": els,
               "host_phases_ms": phases,
               "api": "AcousticModel.forward (host pinned m, eta, wavelet -> host traces)"}
        assert out.shape[0] == args.nt

    peak, peak_kind = measured_peak_hbm()
    roof = None
    if k_n > 0:
        avg_s = k_ms / k_n * 1e-3
        achieved = BYTES_PER_POINT * float(args.n) ** 3 / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": kernel_traffic(args.so), "peak_kind": peak_kind,
                "kernel": "acoustic grid update (%s)" % ("plain" if args.plain else "tiled TMA"),
                "kernel_ms_avg": k_ms / k_n, "kernel_launches_timed": k_n,
                "algorithmic_bytes_per_launch": BYTES_PER_POINT * args.n ** 3,
                "kernel_share_of_step": (k_ms / ms) if ms > 0 else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle._lib()
        v, el = oracle_sample(cfg, args.so, args.cpu_steps)
        cpu = {"value": v, "unit": "GPts/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "%d of %d time steps of the same %d^3 SO%d forward run, FP32 loop nest, %.1f s" % (
                   args.cpu_steps, args.nt, args.n, args.so, el)}
        # the same loop nest on one core, and the FP64 loop nest on all cores
        # (one step each)
        v64, el64 = oracle_sample(cfg, args.so, 1, precision="f64")
        oracle.set_num_threads(1)
        try:
            v1, el1 = oracle_sample(cfg, args.so, 1)
        finally:
            oracle.set_num_threads(None)
        cpu["one_core_f32"] = {"value": v1, "unit": "GPts/s", "cores": 1, "s": el1, "steps": 1}
        cpu["all_cores_f64"] = {"value": v64, "unit": "GPts/s", "cores": oracle.num_threads(), "s": el64,
                                "steps": 1}

    rows = None
    if rank == 0 and not args.no_rows:
        fns = {"diffusion": bench_diffusion, "convection": bench_convection, "laplace": bench_laplace,
               "gradient": bench_gradient, "batched": bench_batched, "learned": bench_learned,
               "two_step": bench_two_step, "space_orders": bench_space_orders}
        rows = {name: fns[name]() for name in args.rows.split(",") if name in fns}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GPts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(config_dict(args), tiling=tiling), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "rows": rows,
                "device": torch.cuda.get_device_name(local)}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
