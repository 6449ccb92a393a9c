"""Pins of the oracle's acoustic forward model with the damping given as a 3-D
field damp[nz][ny][nx] instead of per-axis profiles.

Section "Test case setup" names only "absorbing boundaries with a 10 point
mask"; the API takes either a separable mask (per-axis profiles) or any
non-negative field.  The 3-D path is pinned by what its definition fixes:
a separable field reproduces the per-axis path exactly; the damped scheme is
symmetric for any pointwise damping, so source-receiver reciprocity holds
inside a non-separable sponge (which pins the damped injection scale there);
and the discrete energy does not increase.
"""
import math

import numpy as np

import oracle
import workloads
from tests import fd_exact


def _energy(g, so, dt, m, un1, un):
    """E^{n+1/2} = 1/2 ||(u^{n+1}-u^n)/dt||_m^2 - 1/2 <u^{n+1}, L u^n>."""
    lap = oracle.laplacian(g, so, un)
    return 0.5 * np.sum(m * ((un1 - un) / dt) ** 2) - 0.5 * np.vdot(un1, lap)


def _cfl_bound(so, h, vmax):
    s = fd_exact.second_symbol(so // 2, math.pi)
    return 2.0 / (vmax * math.sqrt(sum(s / hh ** 2 for hh in h)))


def _sponge(shape, h, width, d0, seed):
    """A non-separable absorbing mask: a quadratic ramp in the distance to the
    nearest face (the minimum over the axes, not their sum), times a smooth
    random modulation in [0.5, 1.5]."""
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    edge = np.minimum.reduce([i, nx - 1 - i, j, ny - 1 - j, k, nz - 1 - k]).astype(np.float64)
    ramp = np.clip((width - edge) / width, 0.0, 1.0) ** 2
    mod = workloads.smooth_random(shape, seed, 2.0, 0.5, 1.5)
    return np.ascontiguousarray(d0 * ramp * mod, dtype=np.float32)


def test_separable_field_equals_the_per_axis_profiles_bitwise():
    """Profiles whose sums are exact in FP32 (multiples of 1/64): the 3-D
    field d_x[i] + d_y[j] + d_z[k] gives the per-axis path's result bit for
    bit."""
    shape = (12, 13, 14)
    h = (10.0, 11.0, 9.0)
    rng = np.random.default_rng(1)
    nz, ny, nx = shape
    axes = rng.integers(0, 9, nx + ny + nz).astype(np.float32) / 64.0
    dx, dy, dz = axes[:nx], axes[nx:nx + ny], axes[nx + ny:]
    field = (dz[:, None, None] + dy[None, :, None] + dx[None, None, :]).astype(np.float32)
    assert np.array_equal(field.astype(np.float64),
                          dz[:, None, None].astype(np.float64) + dy[None, :, None] +
                          dx[None, None, :])
    m = workloads.slowness_squared(rng.uniform(1.5, 2.5, shape))
    dt = 0.5 * workloads.cfl_dt(h, 2.5)
    nt = 25
    src = np.array([[[50.0, 61.0, 47.0]]], np.float32)
    rec = np.array([[[20.0, 30.0, 40.0], [100.0, 90.0, 80.0]]], np.float32)
    wav = rng.standard_normal((1, nt, 1)).astype(np.float32)
    u0 = (1e-2 * rng.standard_normal((1, 2) + shape)).astype(np.float32)
    g = oracle.make_grid(shape, h)
    ra, ua = oracle.acoustic_forward(g, 8, dt, nt, m, src, wav, rec, damp=axes, u_init=u0)
    rf, uf = oracle.acoustic_forward(g, 8, dt, nt, m, src, wav, rec, damp=field, u_init=u0,
                                     damp_layout="field")
    np.testing.assert_array_equal(rf, ra)
    np.testing.assert_array_equal(uf, ua)
    assert np.any(field > 0)


def test_reciprocity_inside_a_non_separable_sponge():
    """(m + eta) u+ = dt^2 L u + 2 m u - (m - eta) u- + dt^2 P^T q is symmetric
    for any pointwise eta, so the trace at B from a source at A equals the
    trace at A from a source at B, with A and B inside the sponge where its
    value is not a sum over the axes."""
    shape = (20, 20, 20)
    h = (10.0, 10.0, 10.0)
    g = oracle.make_grid(shape, h)
    m = np.full(shape, np.float32(1 / 2.0 ** 2), dtype=np.float32)
    dt = 0.38 * 10.0 / 2.0
    nt = 40
    damp = _sponge(shape, h, 6, 0.4, 3)
    A = np.array([[[22.3, 81.7, 95.1]]], np.float32)   # x inside the sponge
    B = np.array([[[121.9, 104.4, 11.2]]], np.float32)  # z inside the sponge
    for p in (A, B):
        i, j, k = (p[0, 0] / 10.0).astype(int)
        assert damp[k, j, i] > 0
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None].astype(np.float32)
    rAB, _ = oracle.acoustic_forward(g, 4, dt, nt, m, A, wav, B, damp=damp, damp_layout="field")
    rBA, _ = oracle.acoustic_forward(g, 4, dt, nt, m, B, wav, A, damp=damp, damp_layout="field")
    assert np.max(np.abs(rAB)) > 0
    np.testing.assert_allclose(rAB, rBA, rtol=1e-10, atol=1e-12 * np.max(np.abs(rAB)))


def test_energy_does_not_increase_in_a_non_separable_sponge():
    so = 4
    shape = (16, 16, 16)
    h = (10.0, 10.0, 10.0)
    m = np.full(shape, np.float32(1.0 / 2.0 ** 2), dtype=np.float32)
    dt = 0.8 * _cfl_bound(so, h, 2.0)
    damp = _sponge(shape, h, 5, 0.3, 7)
    g = oracle.make_grid(shape, h)
    u0 = workloads.smooth_random(shape, 8, 2.0, -1, 1).astype(np.float32)
    init = np.stack([u0, u0])[None]
    e = np.zeros((1, 0, 3), np.float32)
    es = []
    for nt in range(2, 50):
        _, uf = oracle.acoustic_forward(g, so, dt, nt, m, e, np.zeros((1, nt, 0), np.float32), e,
                                        damp=damp, u_init=init, damp_layout="field")
        es.append(_energy(g, so, dt, m.astype(np.float64), uf[0, 0], uf[0, 1]))
    d = np.diff(es)
    assert np.all(d <= 1e-12 * es[0])
    assert es[-1] < 0.95 * es[0]
