"""The two-step (temporally blocked) acoustic sweep, through the C ABI.

Both stages of the two-step kernel evaluate the single-step kernel's
expression in the same order on the same values, so a run with 2 steps per
sweep equals a run with 1 bit for bit: both field slots and every receiver
trace, forward and reverse, odd step counts (the last step runs alone),
ragged tiles in every axis, sources fused into both stages.  One run is also
checked against the FP64 oracle at the tolerance of the single-step traces,
and one at the full 512^3 size of the benchmark.
"""
import numpy as np
import pytest

import oracle
from fdrun import AcousticRun, rel_l2
from paper_1707_03776_gb300 import fd
from paper_1707_03776_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-4


def _case(shape, so, nt, seed, nsrc=3, nrec=11):
    h = 10.0
    v = wl.two_layer_velocity(shape, 1500.0, 2500.0)
    m = (1.0 / v ** 2).astype(np.float32)
    sig = wl.sponge_sigma(shape, (h,) * 3, 4, 2500.0, ref_width=40)
    eta = (m.astype(np.float64) * sig).astype(np.float32)
    dt = 0.4 * h / 2500.0
    src = wl.random_points(shape, (h,) * 3, (0, 0, 0), nsrc, seed)
    rec = wl.random_points(shape, (h,) * 3, (0, 0, 0), nrec, seed + 1)
    trace = np.random.default_rng(seed).standard_normal((nt, nsrc)).astype(np.float32)
    return (shape, (h,) * 3, None, so, m, eta, src, trace, rec, nt), dt


def _run(args, dt, k, flags=0, state=None):
    run = AcousticRun(*args, flags=flags)
    fd.fd_operator_set_time_block(run.op.handle, k)
    got_k, ctas = fd.fd_operator_get_time_block(run.op.handle)
    assert got_k == k and ctas > 0
    if state is not None:
        run.set_state(*state)
    run.run(0, args[-1], dt)
    return run


def _slots(run):
    return [run.u.view(s).cpu().numpy().copy() for s in (0, 1)]


@pytest.mark.parametrize("so,shape,nt", [
    (4, (37, 61, 150), 9), (6, (23, 45, 97), 8), (8, (41, 70, 131), 11), (8, (12, 29, 64), 6),
    (8, (3, 33, 70), 5), (8, (16, 16, 16), 4),
])
def test_two_steps_equal_one_bitwise(so, shape, nt):
    args, dt = _case(shape, so, nt, 40 + so)
    state = (wl.random_field(shape, 3, smooth=1), wl.random_field(shape, 4, smooth=1))
    one = _run(args, dt, 1, state=state)
    two = _run(args, dt, 2, state=state)
    for a, b in zip(_slots(one), _slots(two)):
        assert np.abs(a).max() > 0
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(one.rec_trace(), two.rec_trace())


def test_two_steps_reverse_bitwise():
    """FD_FLAG_REVERSE (the adjoint's time loop) pairs steps n, n-1."""
    args, dt = _case((30, 50, 100), 8, 10, 7)
    one = _run(args, dt, 1, flags=fd.FD_FLAG_REVERSE)
    two = _run(args, dt, 2, flags=fd.FD_FLAG_REVERSE)
    for a, b in zip(_slots(one), _slots(two)):
        assert np.abs(a).max() > 0
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(one.rec_trace(), two.rec_trace())


def test_two_steps_match_the_oracle():
    cfg = wl.acoustic_config(n=48, space_order=8, nt=150, sponge=8, nrec_side=9)
    args = (cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"], cfg["src_coords"],
            cfg["src_trace"], cfg["rec_coords"], cfg["nt"])
    run = _run(args, cfg["dt"], 2)
    ou, _, orec = oracle.acoustic_forward(cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["m"], cfg["eta"],
                                          cfg["dt"], cfg["nt"], src_coords=cfg["src_coords"],
                                          src_trace=cfg["src_trace"], rec_coords=cfg["rec_coords"])
    assert np.abs(orec).max() > 0
    assert rel_l2(run.rec_trace(), orec) <= TRACE_TOL
    assert rel_l2(run.state(cfg["nt"])[0], ou) <= TRACE_TOL


def test_two_steps_resume_across_calls():
    """Splitting a run into calls of odd lengths changes which steps pair up,
    not the result."""
    args, dt = _case((20, 40, 80), 8, 17, 11)
    whole = _run(args, dt, 2)
    part = AcousticRun(*args)
    fd.fd_operator_set_time_block(part.op.handle, 2)
    for t0, n in ((0, 3), (3, 5), (8, 9)):
        part.run(t0, n, dt)
    for a, b in zip(_slots(whole), _slots(part)):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(whole.rec_trace(), part.rec_trace())


def test_time_block_errors():
    args, _ = _case((20, 24, 28), 8, 4, 3)
    run = AcousticRun(*args)
    with pytest.raises(fd.FDError):
        fd.fd_operator_set_time_block(run.op.handle, 3)
    plain = AcousticRun(*args, flags=fd.FD_FLAG_PLAIN_KERNELS)
    with pytest.raises(fd.FDError):
        fd.fd_operator_set_time_block(plain.op.handle, 2)
    so16 = AcousticRun(*args[:3], 16, *args[4:])
    with pytest.raises(fd.FDError):
        fd.fd_operator_set_time_block(so16.op.handle, 2)
    assert fd.fd_operator_get_time_block(so16.op.handle)[0] == 1


def test_two_steps_full_size_bitwise():
    """The 512^3 SO8 benchmark workload (one column per SM): 41 steps from
    rest with the Ricker source, both field slots and all 10 201 traces."""
    from paper_1707_03776_gb300.modeling import AcousticModel
    nt = 41
    cfg = wl.acoustic_config(n=512, space_order=8, nt=nt)
    model = AcousticModel(cfg["shape"], cfg["spacing"], cfg["origin"], 8, cfg["src_coords"], cfg["rec_coords"], nt)
    model.load(cfg["m"], cfg["eta"], cfg["src_trace"])
    out = []
    for k in (1, 2):
        fd.fd_operator_set_time_block(model.op.handle, k)
        for s in model.u.slots:
            s.zero_()
        model.rec.data.zero_()
        model.op.apply(0, nt, cfg["dt"])
        model.op.sync()
        out.append([model.u.view(s).cpu().numpy() for s in (0, 1)] + [model.rec.data.cpu().numpy()])
    assert np.abs(out[0][0]).max() > 0 and np.abs(out[0][2]).max() > 0
    for a, b in zip(*out):
        np.testing.assert_array_equal(a, b)


def test_two_steps_bounded_wait_gives_up_and_reports():
    """The failure path of the cooperative launch: tile 0 never receives one
    u^n plane, its bounded wait gives up and records FD_ERR_TIMEOUT, the other
    columns stop waiting on its progress as soon as they see the status, every
    CTA drains the copies it issued, and the next run is exact again."""
    import time
    args, dt = _case((24, 40, 130), 8, 6, 5)
    run = AcousticRun(*args)
    fd.fd_operator_set_time_block(run.op.handle, 2)
    assert fd.fd_operator_get_time_block(run.op.handle)[1] > 1
    fd.fd_operator_debug_stall(run.op.handle, 7)
    t0 = time.perf_counter()
    run.op.apply(0, 4, dt)
    with pytest.raises(fd.FDError) as e:
        run.op.sync()
    assert e.value.status == fd.FD_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    fd.fd_operator_debug_stall(run.op.handle, -1)
    for s in run.u.slots:
        s.zero_()
    run.run(0, 6, dt)
    ref = _run(args, dt, 2)
    for a, b in zip(_slots(run), _slots(ref)):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(run.rec_trace(), ref.rec_trace())
