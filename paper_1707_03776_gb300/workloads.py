"""Seeded synthetic inputs shaped like the paper's workloads.

Both the CUDA path and the CPU oracle consume these arrays; this module holds
none of the method's arithmetic (no stencil, no update, no interpolation).
Everything is generated in FP64 and rounded once to FP32, so that both sides
see bit-identical FP32 inputs.

Axis convention: fields are (n0, n1, n2) row-major with (x, y, z) -> (d0, d1,
d2); z (depth) is the contiguous axis d2 and the surface is z = 0.

Inputs defined here (the readings of the paper's unspecified `Model(...)`):
  * velocity: two layers, 1500 m/s above half depth and 2500 m/s below;
    square slowness m = 1/v^2 (SI units);
  * damping eta = m * sigma with the polynomial sponge
    sigma(x) = sum_axes sigma_max (r/W)^2 on the W cells next to every face
    (r in (0, W] cells into the layer), sigma_max = 3 v_max ln(1/R) / (2 W h),
    R = 1e-3, W = 40 (thinner layers of scaled-down grids keep the 40-cell
    sigma_max); so that dt*eta/m = dt*sigma;
  * source: Ricker wavelet (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2);
  * diffusion: indicator of the ring 0.25 < r < 0.35 about (0.5, 0.5).
"""
import math

import numpy as np

SEED_BASE = 1707_03776


def rng(config_id: int = 0, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + config_id + 1000 * salt)


def ricker(nt: int, dt: float, f0: float = 10.0, t0: float = None) -> np.ndarray:
    """Ricker wavelet sampled at t_n = n dt, n = 0..nt-1 (FP64)."""
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f0 * (t - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def two_layer_velocity(shape, v_top=1500.0, v_bottom=2500.0, interface=None) -> np.ndarray:
    """Velocity (FP64) with v_top for depth index < interface, v_bottom below."""
    nz = shape[-1]
    if interface is None:
        interface = nz // 2
    v = np.full(shape, v_top, dtype=np.float64)
    v[..., interface:] = v_bottom
    return v


def sponge_sigma(shape, spacing, width, v_max, reflection=1e-3, ref_width=None) -> np.ndarray:
    """Polynomial sponge damping rate sigma (1/s, FP64) on every face.

    sigma_max uses `ref_width` cells (default: the layer width); scaled-down
    test grids keep the 40-cell strength so that dt*sigma stays ~0.1 per axis
    (a thin layer with its own sigma_max would push dt*sigma past 1, where the
    explicit damped update is unstable)."""
    sigma = np.zeros(shape, dtype=np.float64)
    if width <= 0:
        return sigma
    ndim = len(shape)
    for a in range(ndim):
        n = shape[a]
        h = spacing[a]
        i = np.arange(n, dtype=np.float64)
        r = np.maximum(0.0, np.maximum(width - i, i - (n - 1 - width)))
        wref = width if ref_width is None else ref_width
        smax = 3.0 * v_max * math.log(1.0 / reflection) / (2.0 * wref * h)
        prof = smax * (r / width) ** 2
        sh = [1] * ndim
        sh[a] = n
        sigma = sigma + prof.reshape(sh)
    return sigma


def acoustic_config(n=512, space_order=8, nt=1000, h=10.0, sponge=40, nrec_side=101,
                    cfl=0.4, v_top=1500.0, v_bottom=2500.0, f0=10.0, ndim=3):
    """The 3D isotropic acoustic forward workload (and its scaled-down copies).

    n^3 interior grid (n^2 in 2D), spacing h, two-layer velocity, `sponge`-cell
    sponge, dt = cfl*h/v_max, one Ricker source at the surface centre just
    below the top sponge, nrec_side^2 receivers on the plane half a cell below
    it (a line of nrec_side receivers in 2D).  Returns a dict of FP32 fields
    and FP64 coordinates.
    """
    shape = (n,) * ndim
    spacing = (h,) * ndim
    origin = (0.0,) * ndim
    v = two_layer_velocity(shape, v_top, v_bottom)
    v_max = max(v_top, v_bottom)
    dt = cfl * h / v_max
    m64 = 1.0 / v ** 2
    m = m64.astype(np.float32)
    sigma = sponge_sigma(shape, spacing, sponge, v_max, ref_width=max(sponge, 40))
    eta = (m.astype(np.float64) * sigma).astype(np.float32)
    depth = float(sponge)
    centre = (n - 1) / 2.0
    if ndim == 3:
        src_idx = np.array([[centre, centre, depth]])
        lo, hi = float(sponge), float(n - 1 - sponge)
        g = np.linspace(lo, hi, nrec_side)
        gx, gy = np.meshgrid(g, g, indexing="ij")
        rec_idx = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, depth + 0.5)], axis=1)
    else:
        src_idx = np.array([[centre, depth]])
        lo, hi = float(sponge), float(n - 1 - sponge)
        g = np.linspace(lo, hi, nrec_side)
        rec_idx = np.stack([g, np.full(g.size, depth + 0.5)], axis=1)
    src_coords = src_idx * h
    rec_coords = rec_idx * h
    src_trace = ricker(nt, dt, f0).astype(np.float32).reshape(nt, 1)
    return dict(shape=shape, spacing=spacing, origin=origin, space_order=space_order,
                m=m, eta=eta, dt=dt, nt=nt, src_coords=src_coords, src_trace=src_trace,
                rec_coords=rec_coords, v_max=v_max)


def diffusion_ring(n=256, a=0.5, nt=500, courant=0.2):
    """2D diffusion workload: n x n nodes at i*h, h = 1/(n-1), the outer rows
    and columns are the zero Dirichlet nodes; u0 = 1 in 0.25 < r < 0.35 about
    (0.5, 0.5).  Returns the full n x n initial field (FP32), the interior
    (n-2) x (n-2) view's parameters and dt = courant*h^2/a."""
    h = 1.0 / (n - 1)
    x = np.arange(n, dtype=np.float64) * h
    X, Y = np.meshgrid(x, x, indexing="ij")
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2
    u0 = ((r2 > 0.25 ** 2) & (r2 < 0.35 ** 2)).astype(np.float32)
    dt = courant * h * h / a
    return dict(u0_full=u0, u0=np.ascontiguousarray(u0[1:-1, 1:-1]), shape=(n - 2, n - 2),
                spacing=(h, h), origin=(h, h), a=a, dt=dt, nt=nt, space_order=2)


def random_field(shape, seed, scale=1.0, smooth=0):
    """Seeded FP32 random field; `smooth` passes of a 3-point box filter per axis."""
    g = np.random.default_rng(SEED_BASE + 7919 * seed)
    u = g.standard_normal(shape)
    for _ in range(smooth):
        for a in range(len(shape)):
            u = (np.roll(u, 1, a) + u + np.roll(u, -1, a)) / 3.0
    return (scale * u).astype(np.float32)


def random_points(shape, spacing, origin, npoint, seed, margin=0.0):
    """Seeded off-grid coordinates inside [origin, origin + (n-1) h] (FP64)."""
    g = np.random.default_rng(SEED_BASE + 104729 * seed)
    ndim = len(shape)
    lo = np.array(origin, dtype=np.float64) + margin * np.array(spacing)
    hi = np.array(origin, dtype=np.float64) + (np.array(shape) - 1 - margin) * np.array(spacing)
    return lo + (hi - lo) * g.random((npoint, ndim))


def random_smooth_velocity(shape, seed, sigma_cells=8.0, vmin=1500.0, vmax=4500.0):
    """Seeded Gaussian-filtered noise rescaled to [vmin, vmax] (FP64)."""
    g = np.random.default_rng(SEED_BASE + 31337 * seed)
    u = g.standard_normal(shape)
    # separable Gaussian filter by FFT along each axis
    for a in range(len(shape)):
        n = shape[a]
        k = np.fft.rfftfreq(n)
        filt = np.exp(-0.5 * (2 * math.pi * k * sigma_cells) ** 2)
        sh = [1] * len(shape)
        sh[a] = filt.size
        u = np.fft.irfft(np.fft.rfft(u, axis=a) * filt.reshape(sh), n=n, axis=a)
    u = (u - u.min()) / (u.max() - u.min())
    return vmin + (vmax - vmin) * u


def gradient_config(n=256, nt=1500, nshots=8, nrec_side=65, h=10.0, space_order=8, sponge=40, f0=10.0):
    """Adjoint/gradient workload: true model two-layer (1500/2500 m/s) plus a
    Gaussian anomaly of +10 % velocity with a 30-cell radius at the centre;
    the starting model is the true background smoothed with a wide Gaussian
    (no anomaly); `nshots` sources on a line at the surface (depth index
    sponge), `nrec_side`^2 receivers half a cell below them; dt at CFL 0.4 of
    the fastest velocity."""
    shape = (n,) * 3
    spacing = (h,) * 3
    v_bg = two_layer_velocity(shape, 1500.0, 2500.0)
    idx = np.arange(n, dtype=np.float64)
    c = (n - 1) / 2.0
    X, Y, Z = np.meshgrid(idx, idx, idx, indexing="ij", sparse=True)
    r2 = (X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2
    v_true = v_bg * (1.0 + 0.10 * np.exp(-r2 / (2.0 * (30.0 / 2.0) ** 2)))
    # smooth starting model: the background convolved with a Gaussian (sigma 10 cells)
    v0 = v_bg.copy()
    k = np.fft.rfftfreq(n)
    filt = np.exp(-0.5 * (2 * math.pi * k * 10.0) ** 2)
    v0 = np.fft.irfft(np.fft.rfft(v0, axis=2) * filt.reshape(1, 1, -1), n=n, axis=2)
    v_max = float(max(v_true.max(), v0.max()))
    dt = 0.4 * h / v_max
    m_true = (1.0 / v_true ** 2).astype(np.float32)
    m0 = (1.0 / v0 ** 2).astype(np.float32)
    sigma = sponge_sigma(shape, spacing, sponge, v_max, ref_width=max(sponge, 40))
    eta = (m0.astype(np.float64) * sigma).astype(np.float32)
    depth = float(sponge)
    xs = np.linspace(sponge + 10.0, n - 1 - sponge - 10.0, nshots)
    shots = [np.array([[x * h, c * h, depth * h]]) for x in xs]
    g = np.linspace(float(sponge), float(n - 1 - sponge), nrec_side)
    gx, gy = np.meshgrid(g, g, indexing="ij")
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, depth + 0.5)], axis=1) * h
    wavelet = ricker(nt, dt, f0).astype(np.float32).reshape(nt, 1)
    return dict(shape=shape, spacing=spacing, origin=(0.0, 0.0, 0.0), space_order=space_order, m_true=m_true,
                m0=m0, eta=eta, dt=dt, nt=nt, shots=shots, wavelet=wavelet, rec_coords=rec)


def batched_config(nshots=64, n_model=512, wmin=160, wmax=320, nt=800, h=10.0, sponge=20, nrec_side=32,
                   f0=10.0, seed=3):
    """Batched-shots workload: a seeded n_model^3 smooth random velocity model
    (Gaussian-filtered noise, sigma 8 cells, 1.5-4.5 km/s, FP32), and `nshots`
    subgrid windows with per-axis sizes uniform in [wmin, wmax] and origins
    uniform such that each window fits.  Every shot has one Ricker source at
    its window's surface centre (depth index `sponge`) and nrec_side^2
    receivers half a cell below; its own `sponge`-cell sponge at the window's
    faces; dt at CFL 0.4 of 4.5 km/s.  Returns the model (FP32 velocity) and a
    list of windows (origin, shape)."""
    g = np.random.default_rng(SEED_BASE + 4242 * seed)
    shape = (n_model,) * 3
    u = g.standard_normal(shape, dtype=np.float32)
    for a in range(3):
        k = np.fft.rfftfreq(n_model).astype(np.float32)
        filt = np.exp(-0.5 * (2 * math.pi * k * 8.0) ** 2).astype(np.float32)
        sh = [1, 1, 1]
        sh[a] = filt.size
        u = np.fft.irfft(np.fft.rfft(u, axis=a) * filt.reshape(sh), n=n_model, axis=a).astype(np.float32)
    lo, hi = float(u.min()), float(u.max())
    v = (1500.0 + 3000.0 * (u - lo) / (hi - lo)).astype(np.float32)
    windows = []
    for _ in range(nshots):
        wshape = tuple(int(x) for x in g.integers(wmin, wmax + 1, size=3))
        origin = tuple(int(g.integers(0, n_model - w + 1)) for w in wshape)
        windows.append((origin, wshape))
    dt = 0.4 * h / 4500.0
    wavelet = ricker(nt, dt, f0).astype(np.float32).reshape(nt, 1)
    return dict(velocity=v, windows=windows, spacing=(h, h, h), dt=dt, nt=nt, sponge=sponge,
                nrec_side=nrec_side, wavelet=wavelet, v_max=4500.0)


def window_shot(cfg, i):
    """Inputs of shot i of a batched_config: m, eta (FP32 window fields),
    source and receiver coordinates in the window's own frame."""
    (o0, o1, o2), shape = cfg["windows"][i]
    v = cfg["velocity"][o0:o0 + shape[0], o1:o1 + shape[1], o2:o2 + shape[2]].astype(np.float64)
    m = (1.0 / v ** 2).astype(np.float32)
    sigma = sponge_sigma(shape, cfg["spacing"], cfg["sponge"], cfg["v_max"], ref_width=40)
    eta = (m.astype(np.float64) * sigma).astype(np.float32)
    h = cfg["spacing"][0]
    depth = float(cfg["sponge"])
    src = np.array([[(shape[0] - 1) / 2.0 * h, (shape[1] - 1) / 2.0 * h, depth * h]])
    n = cfg["nrec_side"]
    gx = np.linspace(depth, shape[0] - 1 - depth, n)
    gy = np.linspace(depth, shape[1] - 1 - depth, n)
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    rec = np.stack([X.ravel(), Y.ravel(), np.full(X.size, depth + 0.5)], axis=1) * h
    return shape, m, eta, src, rec


def layered_velocity(shape, spacing, seed, vmin=1500.0, vmax=3500.0, extent=None):
    """Seeded random layered model (FP64 velocity on the grid's nodes): 3 to 6
    layers below the surface whose interfaces are planes
    z = z_k + s_k x + t_k y with dips of at most ~6 degrees, velocities drawn
    uniform in [vmin, vmax] and sorted to increase with depth.  The model is a
    function of physical position (origin 0, `extent` metres per axis, by
    default the grid's), so grids of different spacing over one extent sample
    the same model."""
    g = np.random.default_rng(SEED_BASE + 7919 * seed)
    ext = [(n - 1) * h for n, h in zip(shape, spacing)] if extent is None else list(extent)
    nl = int(g.integers(3, 7))
    vel = np.sort(g.uniform(vmin, vmax, nl))
    z0 = np.sort(g.uniform(0.15, 0.9, nl - 1)) * ext[2]
    sx = g.uniform(-0.1, 0.1, nl - 1)
    sy = g.uniform(-0.1, 0.1, nl - 1)
    x = np.arange(shape[0]) * spacing[0] - 0.5 * ext[0]
    y = np.arange(shape[1]) * spacing[1] - 0.5 * ext[1]
    z = np.arange(shape[2]) * spacing[2]
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij", sparse=True)
    layer = np.zeros(np.broadcast_shapes(X.shape, Y.shape, Z.shape), dtype=np.int64)
    for k in range(nl - 1):
        layer += (Z >= z0[k] + sx[k] * X + sy[k] * Y).astype(np.int64)
    return vel[layer]


def closure_config(n_coarse=48, nt=400, seed=0, sponge=8, f0=8.0, vmin=1500.0, vmax=3500.0, cfl=0.3,
                   src="random", src_sigma=30.0, nrec_side=None):
    """One learned-closure experiment: the same layered model, source and
    receivers on a coarse grid (n_coarse^3 nodes at 20 m, SO4) and on the fine
    grid whose every other node is a coarse node ((2 n_coarse - 1)^3 at 10 m,
    SO16).  dt_fine = cfl * 10 m / vmax and dt_coarse = 2 dt_fine (the same
    Courant number on both grids); the fine run takes 2 nt steps.

    The source is a Gaussian density (standard deviation `src_sigma` m, cut
    at 2.5 sigma and normalised to unit strength on each grid: sum of density
    times cell volume = 1) times a Ricker wavelet, injected at every node of
    each grid within the cut with amplitude density(node) * wavelet(t)
    (the injection adds amplitude * dt^2/m, so per-node densities discretise
    the same source on both grids).  A smooth source keeps the wavefield free
    of grid-scale content that the coarse grid cannot represent.  The centre
    sits on a coarse node: random in the interior (src="random") or at the
    centre of the top face 6 coarse cells below the sponge (src="surface").
    Receivers: a square lattice of coarse nodes (every other one) on the
    plane 3 coarse cells above the bottom sponge, so that every receiver is
    far from the source and its trace error measures propagation.  Sponges of `sponge` coarse cells
    (twice as many fine cells) with sigma_max of a 400 m layer: the same
    physical profile on both grids."""
    g = np.random.default_rng(SEED_BASE + 104729 * seed + 1)
    hc, hf = 20.0, 10.0
    nc = int(n_coarse)
    nf = 2 * nc - 1
    shape_c, shape_f = (nc,) * 3, (nf,) * 3
    sp_c, sp_f = (hc,) * 3, (hf,) * 3
    ext = [(nc - 1) * hc] * 3
    v_c = layered_velocity(shape_c, sp_c, seed, vmin, vmax, ext)
    v_f = layered_velocity(shape_f, sp_f, seed, vmin, vmax, ext)
    dt_f = cfl * hf / vmax
    dt_c = 2.0 * dt_f

    def fields(v, shape, spacing, width):
        m = (1.0 / v ** 2).astype(np.float32)
        # sigma_max of a 400 m layer on both grids (20 coarse, 40 fine cells)
        sigma = sponge_sigma(shape, spacing, width, vmax, ref_width=20 * width // sponge)
        return m, (m.astype(np.float64) * sigma).astype(np.float32)

    m_c, eta_c = fields(v_c, shape_c, sp_c, sponge)
    m_f, eta_f = fields(v_f, shape_f, sp_f, 2 * sponge)
    reach = int(math.ceil(2.5 * src_sigma / hc))
    lo, hi = sponge + reach + 1, nc - 1 - sponge - reach - 1
    if src == "random":
        s_idx = g.integers(lo, hi + 1, size=3).astype(np.float64)
    else:
        s_idx = np.array([(nc - 1) // 2, (nc - 1) // 2, sponge + 6], dtype=np.float64)
    centre = s_idx * hc

    def gaussian_source(h, n_steps, dt):
        r = int(math.ceil(2.5 * src_sigma / h))
        k = np.arange(-r, r + 1, dtype=np.float64)
        K0, K1, K2 = np.meshgrid(k, k, k, indexing="ij")
        d2 = (K0 ** 2 + K1 ** 2 + K2 ** 2) * h * h
        keep = d2 <= (2.5 * src_sigma) ** 2
        coords = centre + np.stack([K0[keep], K1[keep], K2[keep]], axis=1) * h
        dens = np.exp(-d2[keep] / (2.0 * src_sigma ** 2))
        dens /= dens.sum() * h ** 3  # unit strength on each grid: sum of density * cell volume = 1
        trace = ricker(n_steps, dt, f0)[:, None] * dens[None, :]
        return coords, trace.astype(np.float32)

    src_c, trace_c = gaussian_source(hc, nt, dt_c)
    src_f, trace_f = gaussian_source(hf, 2 * nt, dt_f)
    sub_c = closure_descriptors(v_c, v_f, eta_c, m_c, dt_c, vmax)
    side = np.arange(sponge + 1, nc - sponge - 1, 2, dtype=np.float64)
    if nrec_side is not None:
        side = side[:: max(1, side.size // int(nrec_side))][: int(nrec_side)]
    X, Y = np.meshgrid(side, side, indexing="ij")
    depth = float(nc - 1 - sponge - 3)
    rec_coords = np.stack([X.ravel(), Y.ravel(), np.full(X.size, depth)], axis=1) * hc
    return dict(
        coarse=dict(shape=shape_c, spacing=sp_c, space_order=4, dt=dt_c, nt=nt, m=m_c, eta=eta_c,
                    src_coords=src_c, src_trace=trace_c, sub=sub_c),
        fine=dict(shape=shape_f, spacing=sp_f, space_order=16, dt=dt_f, nt=2 * nt, m=m_f, eta=eta_f,
                  src_coords=src_f, src_trace=trace_f),
        origin=(0.0, 0.0, 0.0), rec_coords=rec_coords, vmax=vmax, vmin=vmin, f0=f0, sponge=sponge, seed=seed,
        src_centre=centre)


def closure_descriptors(v_c, v_f, eta_c, m_c, dt_c, vref):
    """Per-coarse-node descriptors of what the coarse model cannot show (FP32,
    [3, *coarse shape]), from the same model sampled on the fine grid whose
    node 2i is coarse node i, in units of q = v^2 / vref^2:
      0: the full-weighting average of q over the fine nodes of the coarse
         cell (weights 1/4, 1/2, 1/4 per axis) minus q at the coarse node --
         non-zero where an interface crosses the cell;
      1: q(2i, 2j, 2k + 1) - q(2i, 2j, 2k - 1) on the fine grid -- which side
         of the node the interface lies on along the depth axis;
      2: dt sigma, the damping per coarse step (0 outside the sponge).
    Fine indices outside the grid are clamped to its faces."""
    q_f = (np.asarray(v_f, dtype=np.float64) / vref) ** 2
    q_c = (np.asarray(v_c, dtype=np.float64) / vref) ** 2
    nc = q_c.shape
    nf = q_f.shape

    def at(axis, off):
        # fine index 2i + off along `axis`, clamped, for every coarse i
        return np.clip(2 * np.arange(nc[axis]) + off, 0, nf[axis] - 1)

    # the average minus q_c as the weighted sum of differences (weights sum
    # to 1), so that it is exactly 0 where the fine nodes all equal q_c
    dev = np.zeros(nc, dtype=np.float64)
    wts = {-1: 0.25, 0: 0.5, 1: 0.25}
    for o0, w0 in wts.items():
        for o1, w1 in wts.items():
            for o2, w2 in wts.items():
                dev += w0 * w1 * w2 * (q_f[np.ix_(at(0, o0), at(1, o1), at(2, o2))] - q_c)
    dz = q_f[np.ix_(at(0, 0), at(1, 0), at(2, 1))] - q_f[np.ix_(at(0, 0), at(1, 0), at(2, -1))]
    damp = dt_c * np.asarray(eta_c, dtype=np.float64) / np.asarray(m_c, dtype=np.float64)
    return np.stack([dev, dz, damp]).astype(np.float32)


def closure_training_set(count=128, n_coarse=64, nt=600, f0=8.0, first=160, every=40, sponge=8):
    """The closure's training experiments: `count` seeded layered models
    (seeds 0..count-1, random interior sources, `sponge`-cell sponges, or
    with a sequence of widths model s gets width sponge[s % len]) on
    n_coarse^3 coarse grids, and the coarse steps sampled from each fine run:
    every `every` steps from `first` (after the 2/f0 s the source lasts, so
    that the network, which does not see the source, learns the propagation
    error)."""
    widths = [int(sponge)] if np.ndim(sponge) == 0 else [int(w) for w in sponge]
    cfgs = [closure_config(n_coarse, nt, seed=s, f0=f0, sponge=widths[s % len(widths)]) for s in range(count)]
    return cfgs, list(range(first, nt - 2, every))


def smooth_bump(s):
    """C-infinity bump on (0, 1): exp(1 - 1/(1 - (2s-1)^2)), peak 1 at s = 1/2."""
    s = np.asarray(s, dtype=np.float64)
    t = 2.0 * s - 1.0
    out = np.zeros_like(s)
    inside = np.abs(t) < 1.0
    out[inside] = np.exp(1.0 - 1.0 / (1.0 - t[inside] ** 2))
    return out


def convection_config(n=81, c=1.0, courant=0.2, nt=100, extent=2.0):
    """The Linear Convection example: an n x n grid on [0, extent]^2 (x = the
    first axis), velocity c, dt = courant * dx / c, nt steps.  The paper's
    smooth initial condition 1 + b(2x/3) b(2y/3) (its 1D profile is garbled
    in the text; b is the C-infinity bump above) is stored as its deviation
    from the far-field value 1, so that the zero halo is the inflow value."""
    h = extent / (n - 1)
    x = np.arange(n) * h
    w0 = smooth_bump(2.0 * x / 3.0)[:, None] * smooth_bump(2.0 * x / 3.0)[None, :]
    return dict(shape=(n, n), spacing=(h, h), c=c, dt=courant * h / c, nt=nt, u0=w0.astype(np.float32))


def laplace_config(nx=31, ny=31, lx=2.0, ly=1.0, tol=1e-4):
    """The Laplace example: nx x ny nodes on [0, lx] x [0, ly], p = 0
    initially, p = 0 on x = 0 and p = y on x = lx (bc_right), dp/dy = 0 on
    y = 0 and y = ly, stopped when the L1 criterion falls below tol."""
    dx, dy = lx / (nx - 1), ly / (ny - 1)
    p0 = np.zeros((nx, ny), dtype=np.float64)
    p0[-1, :] = np.arange(ny) * dy
    return dict(shape=(nx, ny), spacing=(dx, dy), p0=p0.astype(np.float32), tol=tol)
