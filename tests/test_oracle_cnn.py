"""Pins of the closure network's CPU oracle (CPU only).

  * conv3d equals a brute-force loop over points, taps and channels, and a
    single-channel conv equals scipy.ndimage.correlate with zero padding;
  * input and weight gradients of conv3d equal central finite differences of
    a random linear functional (FP64);
  * the whole network's parameter gradients equal finite differences;
  * bf16_round matches the round-to-nearest-even definition on edge cases;
  * the closure features are linear in the wavefield and equal (u, du, u, du,
    u, du) where the velocity is vref; the restriction keeps coinciding
    nodes; the first Adam step moves every parameter by lr sign(g); the MSE
    gradient matches finite differences; a bias-free ReLU network is
    positively homogeneous (the property the closure relies on).
"""
import itertools

import numpy as np
import pytest

from oracle import cnn


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv_bruteforce():
    x = _rand((5, 4, 6, 3), 1)
    w = _rand((27, 3, 2), 2)
    b = _rand((2,), 3)
    y = cnn.conv3d(x, w, b)
    ref = np.zeros((5, 4, 6, 2))
    for i, j, k in itertools.product(range(5), range(4), range(6)):
        acc = b.copy()
        for t, (a, bb, c) in enumerate(cnn.TAPS):
            ii, jj, kk = i + a, j + bb, k + c
            if 0 <= ii < 5 and 0 <= jj < 4 and 0 <= kk < 6:
                acc += x[ii, jj, kk] @ w[t]
        ref[i, j, k] = acc
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_conv_single_channel_is_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    x = _rand((7, 8, 9), 4)
    k = _rand((3, 3, 3), 5)
    w = k.reshape(27, 1, 1)
    y = cnn.conv3d(x[..., None], w, np.zeros(1))[..., 0]
    ref = ndimage.correlate(x, k, mode="constant", cval=0.0)
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def test_conv_gradients_match_finite_differences():
    x = _rand((4, 5, 3, 2), 6)
    w = _rand((27, 2, 3), 7)
    b = _rand((3,), 8)
    R = _rand((4, 5, 3, 3), 9)  # L = sum(R * y)
    gx = cnn.conv3d_grad_input(R, w)
    gw, gb = cnn.conv3d_grad_weight(x, R)
    L = lambda xx, ww, bbb: float((R * cnn.conv3d(xx, ww, bbb)).sum())  # noqa: E731
    eps = 1e-6
    g = np.random.default_rng(10)
    for _ in range(3):
        dx = g.standard_normal(x.shape)
        fd = (L(x + eps * dx, w, b) - L(x - eps * dx, w, b)) / (2 * eps)
        assert abs(fd - float((gx * dx).sum())) < 1e-7 * max(1.0, abs(fd))
        dw = g.standard_normal(w.shape)
        fd = (L(x, w + eps * dw, b) - L(x, w - eps * dw, b)) / (2 * eps)
        assert abs(fd - float((gw * dw).sum())) < 1e-7 * max(1.0, abs(fd))
    np.testing.assert_allclose(gb, R.reshape(-1, 3).sum(axis=0))


def test_network_gradients_match_finite_differences():
    g = np.random.default_rng(11)
    chans = [3, 4, 4, 4, 1]
    params = [(0.3 * g.standard_normal((27, chans[i], chans[i + 1])), 0.1 * g.standard_normal(chans[i + 1]))
              for i in range(4)]
    x = g.standard_normal((5, 4, 6, 3))
    target = g.standard_normal((5, 4, 6, 1))

    def loss(ps):
        acts, _ = cnn.network_forward(x, ps)
        return 0.5 * float(((acts[-1] - target) ** 2).sum())

    acts, pre = cnn.network_forward(x, params)
    grads = cnn.network_backward(acts, pre, params, acts[-1] - target)
    eps = 1e-6
    for li in range(4):
        dw = g.standard_normal(params[li][0].shape)
        pp = [p for p in params]
        pp[li] = (params[li][0] + eps * dw, params[li][1])
        pm = [p for p in params]
        pm[li] = (params[li][0] - eps * dw, params[li][1])
        fd = (loss(pp) - loss(pm)) / (2 * eps)
        an = float((grads[li][0] * dw).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, fd, an)


def test_bf16_round():
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.1415926, 1e-30, 65504.0], dtype=np.float32)
    r = cnn.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # exactly halfway to 1.0078125: ties to even keeps 1.0
    assert r[2] == np.float32(1.0078125)
    assert r[3] == np.float32(1.0078125)
    assert abs(r[4] - vals[4]) <= 2 ** -8 * abs(vals[4])
    # every result is representable in 8 significand bits
    assert np.all((r.view(np.uint32) & 0xFFFF) == 0)


def test_features_linear_and_reference_velocity():
    g = np.random.default_rng(12)
    u, up = g.standard_normal((3, 4, 5)), g.standard_normal((3, 4, 5))
    vref = 3000.0
    m = np.full((3, 4, 5), 1.0 / vref ** 2)
    f = cnn.features(u, up, m, 2.0, vref)
    for c in range(3):
        np.testing.assert_allclose(f[..., 2 * c], u / 2.0, rtol=1e-14)
        np.testing.assert_allclose(f[..., 2 * c + 1], (u - up) / 2.0, rtol=1e-14, atol=1e-15)
    m2 = np.full((3, 4, 5), 1.0 / (2 * vref) ** 2)  # twice the velocity: q = 4
    f2 = cnn.features(3 * u, 3 * up, m2, 1.0, vref)
    np.testing.assert_allclose(f2[..., 4], 48.0 * u, rtol=1e-13)


def test_features_model_descriptors():
    """Each descriptor s_k adds (s_k u, s_k du) / scale: a descriptor equal to
    1 repeats channels 0 and 1, one equal to q repeats channels 2 and 3, and
    without descriptors the six channels are unchanged."""
    g = np.random.default_rng(13)
    u, up = g.standard_normal((3, 4, 5)), g.standard_normal((3, 4, 5))
    m = 1.0 / (1500.0 + 2000.0 * g.random((3, 4, 5))) ** 2
    vref = 3500.0
    q = 1.0 / (m * vref * vref)
    f0 = cnn.features(u, up, m, 2.0, vref)
    f = cnn.features(u, up, m, 2.0, vref, sub=[np.ones_like(u), q])
    assert f.shape == (3, 4, 5, 10)
    np.testing.assert_array_equal(f[..., :6], f0)
    np.testing.assert_allclose(f[..., 6:8], f0[..., 0:2], rtol=1e-15)
    np.testing.assert_allclose(f[..., 8:10], f0[..., 2:4], rtol=1e-14)


def test_restrict_keeps_coinciding_nodes():
    fine = np.arange(9 * 7 * 5, dtype=np.float64).reshape(9, 7, 5)
    c = cnn.restrict(fine, 2)
    assert c.shape == (5, 4, 3)
    assert c[2, 3, 1] == fine[4, 6, 2]


def test_adam_first_step_and_mse_gradient():
    g = np.random.default_rng(13)
    p = g.standard_normal(50)
    gr = g.standard_normal(50)
    p1, m1, m2 = cnn.adam(p, gr, np.zeros(50), np.zeros(50), 1e-2, 0.9, 0.999, 0.0, 1)
    np.testing.assert_allclose(p1, p - 1e-2 * np.sign(gr), rtol=1e-12)
    pred, res = g.standard_normal(20), g.standard_normal(20)
    loss, gp = cnn.mse_and_grad(pred, res)
    d = g.standard_normal(20)
    eps = 1e-6
    fd = (cnn.mse_and_grad(pred + eps * d, res)[0] - cnn.mse_and_grad(pred - eps * d, res)[0]) / (2 * eps)
    assert abs(fd - float(gp @ d)) < 1e-8


def test_bias_free_network_is_homogeneous():
    g = np.random.default_rng(14)
    chans = [6, 5, 5, 5, 1]
    params = [(g.standard_normal((27, chans[i], chans[i + 1])), np.zeros(chans[i + 1])) for i in range(4)]
    u, up = g.standard_normal((4, 5, 6)), g.standard_normal((4, 5, 6))
    m = np.full((4, 5, 6), 1.0 / 2500.0 ** 2)
    a = cnn.closure_correction(u, up, m, params, 0.5, 3000.0)
    b = cnn.closure_correction(7.5 * u, 7.5 * up, m, params, 0.5, 3000.0)
    np.testing.assert_allclose(b, 7.5 * a, rtol=1e-12, atol=1e-14)
    assert np.all(cnn.closure_correction(0 * u, 0 * up, m, params, 0.5, 3000.0) == 0.0)


def test_splitmix64_published_vector():
    """SplitMix64 against the published first outputs for seed 1234567
    (golden splitmix64.txt), and the unit-variance deviates' range/moments."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    want = [int(line) for line in open(path) if line.strip() and not line.startswith("#")]
    got = [int(cnn.splitmix64(1234567, i)) for i in range(len(want))]
    assert got == want
    xi = cnn.unit_uniform(99, np.arange(200000, dtype=np.uint64))
    assert xi.min() >= -np.sqrt(3.0) and xi.max() < np.sqrt(3.0)
    assert abs(xi.mean()) < 0.01 and abs(xi.var() - 1.0) < 0.01
