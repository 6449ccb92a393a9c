"""Seeded synthetic inputs for the FD wave-propagation sweep.

This module only draws and shapes input data: velocity models, anisotropy
fields, damping profiles, source wavelets and acquisition geometry.  It holds
none of the sweep's arithmetic, and both the CUDA path's tests and the FP64
oracle receive exactly the arrays made here (FP32, rounded once).

The paper's own velocity models are not available; the workloads below stand
in for them with the paper's sizes (512^3 points at 20 m spacing, 1000 ms of
propagation, space orders 4..16; section "Test case setup").

Units: metres, milliseconds, km/s (= m/ms), kHz; m = 1/v^2 in s^2/km^2 (ms^2/m^2).
Arrays are C order [z][y][x]; coordinates are (x, y, z) triples.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

CFL_FACTOR = 0.38  # dt = CFL_FACTOR * h_min / v_max (TTI: / sqrt(1 + 2 eps_max))


@dataclass
class Workload:
    """One forward-modelling problem.  All arrays FP32 and C-contiguous."""

    name: str
    shape: tuple            # (nz, ny, nx), including the damping border
    spacing: tuple          # (hx, hy, hz) in m
    origin: tuple           # (ox, oy, oz) in m
    so: int
    dt: float               # ms
    nt: int
    m: np.ndarray           # [nz][ny][nx] squared slowness
    damp: Optional[np.ndarray]  # [nx + ny + nz] per-axis profiles (1/ms) or None
    src_xyz: np.ndarray     # [nshots][nsrc][3]
    src_wav: np.ndarray     # [nshots][nt][nsrc]
    rec_xyz: np.ndarray     # [nshots][nrec][3]
    nbl: int = 0
    eps: Optional[np.ndarray] = None
    delta: Optional[np.ndarray] = None
    theta: Optional[np.ndarray] = None
    phi: Optional[np.ndarray] = None
    u_init: Optional[np.ndarray] = None  # [nshots][2][nz][ny][nx]
    extra: dict = field(default_factory=dict)

    @property
    def nshots(self):
        return self.src_xyz.shape[0]

    @property
    def npoints(self):
        nz, ny, nx = self.shape
        return nx * ny * nz


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------- velocity models

def two_layer_velocity(shape, v_top=1.5, v_bottom=2.5, interface=None):
    """v = v_top above the interface z-index, v_bottom from it down."""
    nz, ny, nx = shape
    k0 = nz // 2 if interface is None else interface
    v = np.full(shape, v_top, dtype=np.float64)
    v[k0:] = v_bottom
    return v


def smooth_random(shape, seed, sigma, lo, hi):
    """N(0,1) noise (seeded), Gaussian-filtered with std `sigma` grid points via
    FFT in FP64 (periodic), affinely rescaled to [lo, hi]."""
    import scipy.fft as sfft

    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    workers = os.cpu_count() or 1
    spec = sfft.rfftn(noise, workers=workers)
    del noise
    axes_k = []
    for ax, n in enumerate(shape):
        k = sfft.rfftfreq(n) if ax == len(shape) - 1 else sfft.fftfreq(n)
        g = np.exp(-2.0 * (math.pi * sigma * k) ** 2)
        axes_k.append(g)
    spec *= axes_k[0][:, None, None]
    spec *= axes_k[1][None, :, None]
    spec *= axes_k[2][None, None, :]
    f = sfft.irfftn(spec, s=shape, workers=workers)
    del spec
    fmin, fmax = f.min(), f.max()
    f -= fmin
    f *= (hi - lo) / (fmax - fmin)
    f += lo
    return f


def slowness_squared(v):
    return _f32(1.0 / (np.asarray(v, dtype=np.float64) ** 2))


def damping_profile(shape, nbl, spacing, vmax, reflection=1e-3):
    """Per-axis 1-D damping profiles, concatenated [x | y | z].

    Inside the border of width nbl the profile is d0 * (dist/nbl)^2, with dist
    the number of grid points past the border's inner edge and
    d0 = 3 v_max ln(1/R) / (2 nbl h) (the usual quadratic sponge with target
    reflection R).  The damping at (i, j, k) is the sum of the three axes.
    """
    nz, ny, nx = shape
    out = []
    for n, h in ((nx, spacing[0]), (ny, spacing[1]), (nz, spacing[2])):
        d = np.zeros(n, dtype=np.float64)
        if nbl > 0:
            d0 = 3.0 * vmax * math.log(1.0 / reflection) / (2.0 * nbl * h)
            i = np.arange(n)
            dist = np.maximum(np.maximum(nbl - i, i - (n - 1 - nbl)), 0).astype(np.float64)
            d = d0 * (dist / nbl) ** 2
        out.append(d)
    return _f32(np.concatenate(out))


def cfl_dt(spacing, vmax, eps_max=0.0, factor=CFL_FACTOR):
    return factor * min(spacing) / (vmax * math.sqrt(1.0 + 2.0 * eps_max))


def steps_for(t_end, dt):
    """nt = 1 + ceil(T/dt): samples at t = 0, dt, ..., covering [0, T]."""
    return 1 + int(math.ceil(t_end / dt - 1e-12))


# ---------------------------------------------------------------- sources

def ricker(nt, dt, f0=0.010, t0=None, amplitude=1.0):
    """Ricker wavelet q(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
    tau = t - t0, t = n dt (ms, kHz); t0 defaults to 1/f0."""
    t0 = 1.0 / f0 if t0 is None else t0
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f0 * (t - t0)) ** 2
    return amplitude * (1.0 - 2.0 * a) * np.exp(-a)


def random_wavefields(shape, seed, nshots=1, sigma=3.0, amplitude=1.0):
    """Smooth random (u^0, u^-1) pairs [nshots][2][nz][ny][nx] for tests that
    start from a non-zero state."""
    out = np.empty((nshots, 2) + tuple(shape), dtype=np.float32)
    for s in range(nshots):
        for lvl in range(2):
            out[s, lvl] = smooth_random(shape, seed * 101 + 2 * s + lvl, sigma,
                                        -amplitude, amplitude)
    return out


# ---------------------------------------------------------------- workloads

def acoustic_small(so=4, nt=100, seed=0):
    """64^3 (incl. a 10-point border), h = 10 m, two-layer 1.5/2.5 km/s,
    10 Hz Ricker at the grid centre, 64 receivers on a line 20 m below the
    top border."""
    del seed  # fully deterministic recipe
    n, h, nbl = 64, 10.0, 10
    shape = (n, n, n)
    v = two_layer_velocity(shape, 1.5, 2.5, interface=n // 2)
    dt = cfl_dt((h, h, h), 2.5)
    src = np.array([[[31.5 * h, 31.5 * h, 31.5 * h]]], dtype=np.float64)
    xs = np.linspace(10 * h, 53 * h, 64)
    rec = np.stack([xs, np.full(64, 31.5 * h), np.full(64, nbl * h + 20.0)], axis=-1)[None]
    wav = ricker(nt, dt)[None, :, None]
    return Workload("acoustic-64^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v), damping_profile(shape, nbl, (h, h, h), 2.5),
                    _f32(src), _f32(wav), _f32(rec), nbl=nbl)


def acoustic_large(n=512, so=8, t_end=1000.0, nt=None, seed=1, nbl=40, h=20.0,
                   vmin=1.5, vmax=4.5, nshots=1, full_receivers=True):
    """n^3 at h = 20 m, smooth-random velocity in [1.5, 4.5] km/s (seeded noise,
    Gaussian filter sigma = 12 points), 40-point border, one Ricker source at
    (n/2 - 0.5, n/2 - 0.5) h and 20 m below the border, receivers at every
    (x, y) node half a cell below the border."""
    shape = (n, n, n)
    v = smooth_random(shape, seed, 12.0, vmin, vmax)
    dt = cfl_dt((h, h, h), vmax)
    nt = steps_for(t_end, dt) if nt is None else nt
    c = (n / 2 - 0.5) * h
    src = np.tile(np.array([c, c, nbl * h + 20.0]), (nshots, 1, 1))
    if full_receivers:
        gy, gx = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
        rec = np.stack([gx.ravel(), gy.ravel(), np.full(n * n, nbl * h + 0.5 * h)], axis=-1)
    else:
        xs = np.linspace(nbl * h, (n - 1 - nbl) * h, 128)
        rec = np.stack([xs, np.full(128, c), np.full(128, nbl * h + 0.5 * h)], axis=-1)
    rec = np.tile(rec[None], (nshots, 1, 1))
    wav = np.tile(ricker(nt, dt)[None, :, None], (nshots, 1, 1))
    return Workload(f"acoustic-{n}^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v), damping_profile(shape, nbl, (h, h, h), vmax),
                    _f32(src), _f32(wav), _f32(rec), nbl=nbl)


def tti_fields(shape, seeds=(2, 3, 4, 5), sigma=12.0):
    """eps ~ U[0, 0.3], delta ~ U[0, 0.2] then delta <- min(delta, eps) (so that
    eps >= delta everywhere), theta and phi smooth-random in [0, pi/4]."""
    eps = np.random.default_rng(seeds[0]).uniform(0.0, 0.3, shape)
    delta = np.random.default_rng(seeds[1]).uniform(0.0, 0.2, shape)
    delta = np.minimum(delta, eps)
    theta = smooth_random(shape, seeds[2], sigma, 0.0, math.pi / 4)
    phi = smooth_random(shape, seeds[3], sigma, 0.0, math.pi / 4)
    return _f32(eps), _f32(delta), _f32(theta), _f32(phi)


def tti_large(n=512, so=8, t_end=1000.0, nt=None, nbl=40, h=20.0, velocity="two-layer",
              nshots=1, full_receivers=True, sigma=12.0):
    """TTI at n^3: two-layer 1.5/2.5 km/s (or smooth-random 1.5..4.5), eps/delta
    uniform, theta/phi smooth, source and receivers as in `acoustic_large`."""
    shape = (n, n, n)
    if velocity == "two-layer":
        v = two_layer_velocity(shape, 1.5, 2.5)
        vmax = 2.5
    else:
        v = smooth_random(shape, 1, sigma, 1.5, 4.5)
        vmax = 4.5
    eps, delta, theta, phi = tti_fields(shape, sigma=sigma)
    dt = cfl_dt((h, h, h), vmax, eps_max=float(eps.max()))
    nt = steps_for(t_end, dt) if nt is None else nt
    c = (n / 2 - 0.5) * h
    src = np.tile(np.array([c, c, nbl * h + 20.0]), (nshots, 1, 1))
    if full_receivers:
        gy, gx = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
        rec = np.stack([gx.ravel(), gy.ravel(), np.full(n * n, nbl * h + 0.5 * h)], axis=-1)
    else:
        xs = np.linspace(nbl * h, (n - 1 - nbl) * h, 128)
        rec = np.stack([xs, np.full(128, c), np.full(128, nbl * h + 0.5 * h)], axis=-1)
    rec = np.tile(rec[None], (nshots, 1, 1))
    wav = np.tile(ricker(nt, dt)[None, :, None], (nshots, 1, 1))
    return Workload(f"tti-{n}^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v), damping_profile(shape, nbl, (h, h, h), vmax),
                    _f32(src), _f32(wav), _f32(rec), nbl=nbl, eps=eps, delta=delta,
                    theta=theta, phi=phi)


def tti_small(so=4, nt=100, n=48, h=10.0, nbl=8, seed=7):
    """Small TTI case for parity: two-layer velocity, anisotropy as tti_fields
    (smoothing sigma = 4 points), off-node source at the centre."""
    shape = (n, n, n)
    v = two_layer_velocity(shape, 1.5, 2.5)
    eps, delta, theta, phi = tti_fields(shape, seeds=(seed, seed + 1, seed + 2, seed + 3),
                                        sigma=4.0)
    dt = cfl_dt((h, h, h), 2.5, eps_max=float(eps.max()))
    c = (n / 2 - 0.5) * h
    src = np.array([[[c, c, c]]])
    xs = np.linspace(nbl * h, (n - 1 - nbl) * h, 32)
    rec = np.stack([xs, np.full(32, c), np.full(32, nbl * h + 20.0)], axis=-1)[None]
    wav = ricker(nt, dt, f0=0.015)[None, :, None]
    return Workload(f"tti-{n}^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v), damping_profile(shape, nbl, (h, h, h), 2.5),
                    _f32(src), _f32(wav), _f32(rec), nbl=nbl, eps=eps, delta=delta,
                    theta=theta, phi=phi)


def fwi_layered(n=256, so=8, nt=2000, nshots=16, h=20.0, nbl=40, receivers_per_side=None,
                smooth_sigma=10.0, f0=0.010):
    """FWI gradient problem: a 4-layer true model (1.5, 2.0, 2.75, 3.5 km/s,
    equal thicknesses below the top border), the initial model is the true one
    Gaussian-smoothed (sigma = 10 points); shots on a 4 x 4 grid 20 m below the
    top border; receivers on a full surface grid half a cell below the border.
    Returns (true, initial) Workloads sharing the geometry."""
    shape = (n, n, n)
    v = np.empty(shape, dtype=np.float64)
    layers = (1.5, 2.0, 2.75, 3.5)
    edges = np.linspace(nbl, n, len(layers) + 1).astype(int)
    v[: edges[1]] = layers[0]
    for i, vel in enumerate(layers):
        v[edges[i]:edges[i + 1]] = vel
    # the model varies with depth only, so the 3-D Gaussian smoothing is the
    # 1-D smoothing of the depth profile (edges held constant, no wrap)
    from scipy.ndimage import gaussian_filter1d
    prof0 = gaussian_filter1d(v[:, 0, 0], smooth_sigma, mode="nearest")
    v0 = np.broadcast_to(prof0[:, None, None], shape).copy()
    vmax = max(layers)
    dt = cfl_dt((h, h, h), vmax)
    side = int(round(math.sqrt(nshots)))
    xs = np.linspace(nbl * h, (n - 1 - nbl) * h, side + 2)[1:-1]
    sx, sy = np.meshgrid(xs, xs, indexing="ij")
    src = np.stack([sx.ravel(), sy.ravel(), np.full(side * side, nbl * h + 20.0)], -1)[:, None, :]
    r = n if receivers_per_side is None else receivers_per_side
    gx = np.linspace(0.0, (n - 1) * h, r)
    gy, gx = np.meshgrid(gx, gx, indexing="ij")
    rec = np.stack([gx.ravel(), gy.ravel(), np.full(r * r, nbl * h + 0.5 * h)], -1)
    rec = np.tile(rec[None], (src.shape[0], 1, 1))
    wav = np.tile(ricker(nt, dt, f0=f0)[None, :, None], (src.shape[0], 1, 1))
    damp = damping_profile(shape, nbl, (h, h, h), vmax)
    true = Workload(f"fwi-true-{n}^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v), damp, _f32(src), _f32(wav), _f32(rec), nbl=nbl)
    init = Workload(f"fwi-init-{n}^3", shape, (h, h, h), (0.0, 0.0, 0.0), so, dt, nt,
                    slowness_squared(v0), damp, _f32(src), _f32(wav), _f32(rec), nbl=nbl)
    return true, init
