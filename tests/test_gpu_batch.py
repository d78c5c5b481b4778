"""Batches of shots (fd_batch_*): one launch per step for all shots.

Each shot is an ordinary acoustic operator on its own grid; advancing them
together in a batch (eager launches, and a captured CUDA graph replayed) must
give bit-identical fields and traces to advancing each operator alone, since
every grid point sees the same arithmetic.  One shot is also checked against
the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from fdrun import AcousticRun, rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _shots(nt):
    out = []
    for i, n in enumerate([(40, 52, 70), (36, 60, 64), (52, 33, 90), (30, 30, 30)]):
        cfg = wl.acoustic_config(n=1, space_order=8, nt=nt, sponge=6, nrec_side=6)
        shape = n
        h = (10.0,) * 3
        v = wl.random_smooth_velocity(shape, 10 + i, sigma_cells=4.0, vmin=1500.0, vmax=4500.0)
        m = (1.0 / v ** 2).astype(np.float32)
        sig = wl.sponge_sigma(shape, h, 6, 4500.0, ref_width=40)
        eta = (m.astype(np.float64) * sig).astype(np.float32)
        dt = 0.4 * 10.0 / 4500.0
        src = np.array([[shape[0] / 2 * 10.0, shape[1] / 2 * 10.0, 60.0]])
        gx = np.linspace(60.0, (shape[0] - 7) * 10.0, 7)
        rec = np.stack([gx, np.full(7, shape[1] * 5.0), np.full(7, 65.0)], axis=1)
        wav = wl.ricker(nt, dt, 20.0).astype(np.float32).reshape(nt, 1)
        out.append((shape, h, m, eta, dt, src, wav, rec))
    return out


def _make(shot, nt):
    shape, h, m, eta, dt, src, wav, rec = shot
    return AcousticRun(shape, h, None, 8, m, eta, src, wav, rec, nt)


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_batch_equals_individual_runs(graph):
    nt = 60
    shots = _shots(nt)
    dt = shots[0][4]
    alone = []
    for sh in shots:
        run = _make(sh, nt)
        run.run(0, nt, dt)
        alone.append((run.state(nt)[0], run.rec_trace()))
    runs = [_make(sh, nt) for sh in shots]
    batch = fd.Batch([r.op for r in runs], rows=12, stages=3)
    rows, stages, ctas, _ = batch.info()
    assert rows <= 12 and stages == 3 and ctas > 0
    if graph:
        batch.capture(0, nt, dt)
        batch.replay()
    else:
        batch.apply(0, 20, dt)
        batch.apply(20, nt - 20, dt)
    batch.sync()
    assert batch.info()[3] == nt
    for run, (u_ref, rec_ref) in zip(runs, alone):
        np.testing.assert_array_equal(run.state(nt)[0], u_ref)
        np.testing.assert_array_equal(run.rec_trace(), rec_ref)
    # and one shot against the FP64 oracle
    shape, h, m, eta, dt, src, wav, rec = shots[2]
    _, _, orec = oracle.acoustic_forward(shape, h, (0, 0, 0), 8, m, eta, dt, nt, src_coords=src, src_trace=wav,
                                         rec_coords=rec)
    assert rel_l2(runs[2].rec_trace(), orec) <= 1e-4


def test_batch_rejects_mismatched_operators():
    nt = 10
    shots = _shots(nt)
    a = _make(shots[0], nt)
    shape, h, m, eta, dt, src, wav, rec = shots[1]
    b = AcousticRun(shape, h, None, 4, m, eta, src, wav, rec, nt)
    with pytest.raises(fd.FDError) as e:
        fd.Batch([a.op, b.op])
    assert e.value.status == fd.FD_ERR_UNSUPPORTED
    c = AcousticRun(shape, h, None, 8, m, eta, src, wav, rec, nt, flags=fd.FD_FLAG_REVERSE)
    with pytest.raises(fd.FDError):
        fd.Batch([a.op, c.op])


def test_batch_autotune_picks_a_tiling_and_keeps_results_bitwise():
    """fd_batch_autotune times tile heights x depths on the batch's own data
    and keeps the fastest; the tiling changes no result bit, so after tuning
    (and after forcing another tiling) the batch still reproduces the
    individual runs exactly."""
    nt = 40
    shots = _shots(nt)
    dt = shots[0][4]
    alone = []
    for sh in shots:
        run = _make(sh, nt)
        run.run(0, nt, dt)
        alone.append((run.state(nt)[0], run.rec_trace()))
    runs = [_make(sh, nt) for sh in shots]
    batch = fd.Batch([r.op for r in runs], rows=30, stages=2)
    rows, stages, ms = batch.autotune(0, 10, dt)
    assert 10 <= rows <= 30 and 2 <= stages <= 4 and ms > 0
    info = batch.info()
    assert info[1] == stages and info[0] <= rows and info[2] > 0
    for tiling in ("tuned", "forced"):
        if tiling == "forced":
            other = (10, 2) if (rows, stages) != (10, 2) else (16, 3)
            batch = fd.Batch([r.op for r in runs], rows=other[0], stages=other[1])
        for r in runs:
            for s in r.u.slots:
                s.zero_()
            r.rec.data.zero_()
        batch.apply(0, nt, dt)
        batch.sync()
        for run, (u_ref, rec_ref) in zip(runs, alone):
            np.testing.assert_array_equal(run.state(nt)[0], u_ref)
            np.testing.assert_array_equal(run.rec_trace(), rec_ref)


@pytest.mark.parametrize("so,rows,stages", [(4, 12, 3), (16, 10, 2)])
def test_batch_sweeps_several_columns_per_cta(so, rows, stages):
    """More tile columns than CTAs, so that each persistent CTA sweeps two or
    three columns in a row with its ring positions running on from one column
    to the next (the producer warp fetches the next column while the compute
    warps finish the last): fields and traces still equal the individual runs
    bit for bit, at a low and the highest space order."""
    nt = 24
    h = (10.0,) * 3
    dt = 0.3 * 10.0 / 4500.0
    shots = []
    for i, shape in enumerate([(48, 144, 320), (40, 150, 300), (56, 130, 256)] * 6):
        v = wl.random_smooth_velocity(shape, 40 + i, sigma_cells=4.0, vmin=1500.0, vmax=4500.0)
        m = (1.0 / v ** 2).astype(np.float32)
        eta = (m.astype(np.float64) * wl.sponge_sigma(shape, h, 6, 4500.0, ref_width=40)).astype(np.float32)
        src = np.array([[shape[0] * 5.0, shape[1] * 5.0, 60.0 + 10.0 * i]])
        gx = np.linspace(60.0, (shape[0] - 7) * 10.0, 5)
        rec = np.stack([gx, np.full(5, shape[1] * 5.0), np.full(5, 75.0)], axis=1)
        wav = wl.ricker(nt, dt, 25.0).astype(np.float32).reshape(nt, 1)
        shots.append((shape, m, eta, src, wav, rec))
    alone = []
    for shape, m, eta, src, wav, rec in shots:
        run = AcousticRun(shape, h, None, so, m, eta, src, wav, rec, nt)
        run.run(0, nt, dt)
        alone.append((run.state(nt)[0], run.rec_trace()))
        del run
    runs = [AcousticRun(shape, h, None, so, m, eta, src, wav, rec, nt) for shape, m, eta, src, wav, rec in shots]
    batch = fd.Batch([r.op for r in runs], rows=rows, stages=stages)
    r_used, _, ctas, _ = batch.info()
    columns = sum(-(-s[0][1] // r_used) * -(-s[0][2] // 64) for s in shots)
    assert columns >= 2 * ctas, (columns, ctas)
    batch.apply(0, nt, dt)
    batch.sync()
    for run, (u_ref, rec_ref) in zip(runs, alone):
        np.testing.assert_array_equal(run.state(nt)[0], u_ref)
        np.testing.assert_array_equal(run.rec_trace(), rec_ref)


def test_batch_mixed_and_degenerate_shots():
    """Shots without sources, without receivers, and on degenerate windows
    (a few planes, rows or columns; ragged against the 64-column tiles) in one
    batch: every shot's field and traces equal its individual run bit for
    bit."""
    nt = 30
    h = (10.0,) * 3
    dt = 0.3 * 10.0 / 4500.0
    specs = [((5, 6, 7), True, True), ((2, 33, 64), True, False), ((40, 52, 70), False, True),
             ((17, 3, 130), True, True), ((9, 40, 5), False, False)]
    shots = []
    for i, (shape, with_src, with_rec) in enumerate(specs):
        v = wl.random_smooth_velocity(shape, 60 + i, sigma_cells=2.0, vmin=1500.0, vmax=4500.0)
        m = (1.0 / v ** 2).astype(np.float32)
        eta = (m.astype(np.float64) * wl.sponge_sigma(shape, h, 1, 4500.0, ref_width=40)).astype(np.float32)
        ext = [(n - 1) * 10.0 for n in shape]
        src = np.array([[0.5 * ext[0], 0.5 * ext[1], 0.4 * ext[2]]]) if with_src else None
        wav = wl.ricker(nt, dt, 25.0).astype(np.float32).reshape(nt, 1) if with_src else None
        rec = wl.random_points(shape, h, (0.0,) * 3, 7, 80 + i) if with_rec else None
        shots.append((shape, m, eta, src, wav, rec))

    def make(sh):
        shape, m, eta, src, wav, rec = sh
        return AcousticRun(shape, h, None, 8, m, eta, src, wav, rec, nt)

    tiled = []
    for sh in shots:
        r = make(sh)
        if fd.fd_operator_get_tiling(r.op.handle)[0] > 0:
            tiled.append(sh)
        del r
    assert len(tiled) >= 4, [s[0] for s in tiled]
    alone = []
    for sh in tiled:
        run = make(sh)
        run.run(0, nt, dt)
        alone.append((run.state(nt)[0], run.rec_trace() if sh[5] is not None else None))
    runs = [make(sh) for sh in tiled]
    batch = fd.Batch([r.op for r in runs], rows=12, stages=3)
    batch.apply(0, nt, dt)
    batch.sync()
    for run, (u_ref, rec_ref) in zip(runs, alone):
        np.testing.assert_array_equal(run.state(nt)[0], u_ref)
        if rec_ref is not None:
            np.testing.assert_array_equal(run.rec_trace(), rec_ref)
