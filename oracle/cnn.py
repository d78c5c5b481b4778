"""CPU oracle for the learned closure's 3D CNN (test infrastructure only).

Plain FP64 numpy restatement of what the closure network computes; the CUDA
implicit-GEMM kernels are checked against it.  Only the test suite and the
benchmark may import it.

Conventions (channels-last, as the device stores activations):
  x   [n0, n1, n2, C_in]           input field
  w   [27, C_in, C_out]            kernel taps; tap t = (a+1)*9 + (b+1)*3 + (c+1)
                                   for offsets a, b, c in {-1, 0, 1}
  b   [C_out]                      bias
  y[i,j,k,o] = b[o] + sum_t sum_c w[t, c, o] x[i+a, j+b, k+c, c]
  with x = 0 outside the grid (zero padding, output the same size): a
  3x3x3 cross-correlation.

The network: conv(C0 -> 16) ReLU, conv(16 -> 16) ReLU, conv(16 -> 16) ReLU,
conv(16 -> 1), no biases; the closure adds rho times its output to the coarse
update.  Also here: the closure's input features, the fine-to-coarse
injection, the training loss and Adam (Kingma and Ba 2015, Algorithm 1).
"""
import math

import numpy as np

TAPS = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]


def _shift(x, a, b, c):
    """x shifted so that out[i,j,k] = x[i+a, j+b, k+c], zero outside."""
    out = np.zeros_like(x)
    n0, n1, n2 = x.shape[:3]
    src = (slice(max(a, 0), n0 + min(a, 0)), slice(max(b, 0), n1 + min(b, 0)), slice(max(c, 0), n2 + min(c, 0)))
    dst = (slice(max(-a, 0), n0 + min(-a, 0)), slice(max(-b, 0), n1 + min(-b, 0)),
           slice(max(-c, 0), n2 + min(-c, 0)))
    out[dst] = x[src]
    return out


def conv3d(x, w, b):
    """y = b + sum over taps of shifted x times the tap's C_in x C_out matrix."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[2],), dtype=np.float64)
    y += np.asarray(b, dtype=np.float64)
    for t, (a, bb, c) in enumerate(TAPS):
        y += _shift(x, a, bb, c) @ w[t]
    return y


def conv3d_grad_input(gy, w):
    """dL/dx for y = conv3d(x, w, b): gx[p] = sum_t w[t] gy[p - offset_t]."""
    gy = np.asarray(gy, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    gx = np.zeros(gy.shape[:3] + (w.shape[1],), dtype=np.float64)
    for t, (a, bb, c) in enumerate(TAPS):
        gx += _shift(gy, -a, -bb, -c) @ w[t].T
    return gx


def conv3d_grad_weight(x, gy):
    """(dL/dw, dL/db): gw[t] = sum_p x[p + offset_t]^T gy[p], gb = sum_p gy[p]."""
    x = np.asarray(x, dtype=np.float64)
    gy = np.asarray(gy, dtype=np.float64)
    cin, cout = x.shape[3], gy.shape[3]
    gw = np.zeros((27, cin, cout), dtype=np.float64)
    G = gy.reshape(-1, cout)
    for t, (a, bb, c) in enumerate(TAPS):
        gw[t] = _shift(x, a, bb, c).reshape(-1, cin).T @ G
    return gw, G.sum(axis=0)


def network_forward(x, params, store=None):
    """Activations of the 4-layer network; params = [(w, b)] * 4 (b may be
    zeros: the closure's network has none).  `store` (optional) maps every
    hidden activation to the precision it is stored in between layers (the
    device keeps them in BF16: store=bf16_round); the output stays FP64."""
    acts = [np.asarray(x, dtype=np.float64)]
    pre = []
    h = acts[0]
    for li, (w, b) in enumerate(params):
        z = conv3d(h, w, b)
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        if store is not None and li < len(params) - 1:
            h = np.asarray(store(h), dtype=np.float64)
        acts.append(h)
    return acts, pre


def network_backward(acts, pre, params, gout, store=None):
    """Gradients of a scalar loss with dL/d(output) = gout: [(gw, gb)] per layer.
    `store` (optional) maps every stored gradient dL/dh (gout included) to its
    storage precision, as network_forward's does for activations; the ReLU
    derivative is taken from the stored activation (h > 0), which equals z > 0
    for FP64 storage."""
    grads = [None] * len(params)
    rnd = (lambda a: a) if store is None else (lambda a: np.asarray(store(a), dtype=np.float64))
    g = rnd(np.asarray(gout, dtype=np.float64))
    for li in range(len(params) - 1, -1, -1):
        gw, gb = conv3d_grad_weight(acts[li], g)
        grads[li] = (gw, gb)
        if li > 0:
            g = rnd(conv3d_grad_input(g, params[li][0]) * (acts[li] > 0.0))
    return grads


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)


def features(u, u_prev, m, scale, vref, sub=()):
    """Closure inputs [n0, n1, n2, 6 + 2 len(sub)]: with du = u - u_prev and
    q = 1/(m vref^2), (u, du, q u, q du, q^2 u, q^2 du) / scale, then for each
    model descriptor s_k in `sub` (fields of u's shape) (s_k u, s_k du) / scale."""
    u = np.asarray(u, dtype=np.float64)
    du = u - np.asarray(u_prev, dtype=np.float64)
    q = 1.0 / (np.asarray(m, dtype=np.float64) * vref * vref)
    ch = [u, du, q * u, q * du, q * q * u, q * q * du]
    for s_k in sub:
        s_k = np.asarray(s_k, dtype=np.float64)
        ch += [s_k * u, s_k * du]
    return np.stack(ch, axis=-1) / scale


def splitmix64(key, counter):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) output for state
    key + (counter + 1) * 0x9E3779B97F4A7C15 (uint64 arrays)."""
    M = np.uint64(0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (np.uint64(key) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)) & M
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & M
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & M
    return z ^ (z >> np.uint64(31))


def unit_uniform(key, counter):
    """Unit-variance uniform deviates sqrt(3) (2 r - 1), r = top 24 bits / 2^24."""
    r = (splitmix64(key, counter) >> np.uint64(40)).astype(np.float64) / 16777216.0
    return math.sqrt(3.0) * (2.0 * r - 1.0)


def noisy_states(u, u_prev, noise, seed):
    """The training-time perturbation of the closure's input states: point p
    (dense index) gets noise * xi(2p) and noise * xi(2p + 1)."""
    p = np.arange(np.asarray(u).size, dtype=np.uint64).reshape(np.shape(u))
    return (np.asarray(u, dtype=np.float64) + noise * unit_uniform(seed, 2 * p),
            np.asarray(u_prev, dtype=np.float64) + noise * unit_uniform(seed, 2 * p + np.uint64(1)))


def restrict(fine, factor):
    """Coarse field whose node i is fine node factor*i on every axis."""
    return np.asarray(fine)[::factor, ::factor, ::factor]


def mse_and_grad(pred, residual):
    """(mean (pred - residual)^2, its gradient with respect to pred)."""
    e = np.asarray(pred, dtype=np.float64) - np.asarray(residual, dtype=np.float64)
    return float((e * e).mean()), 2.0 * e / e.size


def adam(params, grads, m1, m2, lr, beta1, beta2, eps, step):
    """One Adam update (step counts from 1); returns new (params, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * grads
    m2 = beta2 * m2 + (1.0 - beta2) * grads * grads
    mhat = m1 / (1.0 - beta1 ** step)
    vhat = m2 / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m1, m2


def closure_correction(u, u_prev, m, params, rho, vref):
    """rho * network(features(u^n, u^{n-1})): the term the learned closure
    adds to the coarse update (scale 1: the network is homogeneous)."""
    acts, _ = network_forward(features(u, u_prev, m, 1.0, vref), params)
    return rho * acts[-1][..., 0]
