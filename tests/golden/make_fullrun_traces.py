"""Write the expected values of the full-run parity gate from the FP64 oracle.

The gate is the forward operator of the paper's Seismic Inversion Example run
for the whole configured time on the 512^3 two-layer model (10 m, 40-cell
sponge, one 10 Hz Ricker source at the surface centre, 101 x 101 receivers,
dt at CFL 0.4, 1000 steps).  This script calls only the oracle (`oracle/`,
FP64 loop nest) and the seeded input generator; nothing here runs on a GPU
and no value comes from the CUDA path.

What it stores (`fullrun_<n>_so<SO>_nt<nt>.npz`):
  * `rec_index`  -- a fixed, seeded subset of the receivers (int32);
  * `traces`     -- their FP64 oracle traces rec[n][p], n = 0..nt-1, stored
                    rounded to FP32 (the 1e-4 trace tolerance is 1000 times
                    the FP32 rounding of the stored value);
  * `field_sub`  -- u^{nt} on every 8th node along each axis, FP32-rounded;
  * `field_norm` -- ||u^{nt}||_2 over the whole grid, FP64;
  * the workload's sizes, so that the test can check it runs the same case.

The FP64 run needs about 7 GB of host memory at 512^3 and 1-2 hours of eight
cores per space order.  Usage:

    python tests/golden/make_fullrun_traces.py --so 8 [--n 512 --nt 1000]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1707_03776_gb300 import workloads as wl  # noqa: E402

NREC_KEEP = 512
FIELD_STRIDE = 8


def golden_path(n, so, nt):
    return os.path.join(HERE, "fullrun_%d_so%d_nt%d.npz" % (n, so, nt))


def receiver_subset(nrec, keep, so):
    rng = np.random.default_rng(1707_03776 + 100 * so)
    return np.sort(rng.choice(nrec, size=min(keep, nrec), replace=False)).astype(np.int32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--so", type=int, default=8)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nt", type=int, default=1000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    cfg = wl.acoustic_config(n=a.n, space_order=a.so, nt=a.nt)
    idx = receiver_subset(cfg["rec_coords"].shape[0], NREC_KEEP, a.so)
    t = time.time()
    uc, _, rt = oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], a.so, cfg["m"], cfg["eta"],
                                        cfg["dt"], cfg["nt"], src_coords=cfg["src_coords"],
                                        src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"][idx],
                                        precision="f64")
    secs = time.time() - t
    out = a.out or golden_path(a.n, a.so, a.nt)
    s = FIELD_STRIDE
    np.savez_compressed(out, rec_index=idx, traces=rt.astype(np.float32),
                        field_sub=uc[::s, ::s, ::s].astype(np.float32), field_stride=np.int32(s),
                        field_norm=np.float64(np.linalg.norm(uc)), n=np.int32(a.n), so=np.int32(a.so),
                        nt=np.int32(a.nt), dt=np.float64(cfg["dt"]), oracle_seconds=np.float64(secs))
    print("wrote %s (%.0f s of FP64 oracle, |u|=%.6e, max|trace|=%.3e)"
          % (out, secs, np.linalg.norm(uc), np.abs(rt).max()))


if __name__ == "__main__":
    main()
