"""Pins of the oracle's alternative TTI readings: staggered first derivatives
(inner D+, outer D-) and receivers recording (p + r)/2.

The rotated operators of the paper's TTI test case (section "Test case
setup") are built from first-derivative operators; the paper does not say
whether these are centred or staggered, nor which field the receivers record.
The oracle implements both alternatives; these tests pin them against exact
rational weights, the closed-form plane-wave symbols, the adjoint pairing of
D+ and D-, and the isotropic limit.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests import fd_exact


def grid(shape, h=(1.0, 1.0, 1.0), o=(0.0, 0.0, 0.0)):
    return oracle.make_grid(shape, h, o)


def coords(shape, h, o=(0.0, 0.0, 0.0)):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) * h[2] + o[2], np.arange(ny) * h[1] + o[1],
                          np.arange(nx) * h[0] + o[0], indexing="ij")
    return x, y, z


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6, 7, 8])
def test_staggered_weights_match_exact_moment_solution(r):
    exact = [float(v) for v in fd_exact.staggered_weights(r)]
    np.testing.assert_allclose(oracle.staggered_weights(r), exact, rtol=1e-14, atol=0)


def test_staggered_weights_radius2_known_values():
    np.testing.assert_allclose(oracle.staggered_weights(2), [0.0, 9 / 8, -1 / 24], rtol=1e-15)


@pytest.mark.parametrize("so", [2, 4, 8, 16])
@pytest.mark.parametrize("kind,shift", [("forward", 0.5), ("backward", -0.5)])
def test_staggered_derivative_exact_on_polynomials(so, kind, shift):
    """D+ f at node i is f' at i + 1/2 and D- f is f' at i - 1/2, exactly for
    polynomials of degree <= so and not for degree so + 1 (checked at the
    centre node, x = 0.3, of a line long enough for the stencil)."""
    r = so // 2
    h = 0.5
    n = 2 * r + 5
    ic = n // 2
    shape = (3, 3, n)
    x0 = 0.3 - ic * h
    x, _, _ = coords(shape, (h, 1.0, 1.0), (x0, 0.0, 0.0))
    g = grid(shape, (h, 1.0, 1.0), (x0, 0.0, 0.0))
    a = oracle.staggered_weights(r)
    for p in range(0, so + 2):
        f = x ** p
        d = oracle.first_derivative(g, so, 0, f, kind=kind)[1, 1, ic]
        xe = 0.3 + shift * h
        d_exact = p * xe ** (p - 1) if p >= 1 else 0.0
        # rounding bound: the stencil sums |a_k| |f| over nodes within r h
        fmax = max(abs(0.3 - (r + 1) * h), abs(0.3 + (r + 1) * h)) ** p
        tol = 1e-14 * 2 * np.sum(np.abs(a)) * fmax / h
        if p <= so:
            assert abs(d - d_exact) <= tol + 1e-13, (p, d, d_exact)
        else:
            assert abs(d - d_exact) > 1e3 * tol + 1e-6, (p, d, d_exact)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_staggered_pair_is_negative_transpose(axis):
    """<D+ f, g> = -<f, D- g> on the Dirichlet grid (zero ghosts)."""
    shape = (9, 10, 11)
    g = grid(shape, (0.7, 1.3, 0.9))
    rng = np.random.default_rng(31 + axis)
    f = rng.standard_normal(shape)
    q = rng.standard_normal(shape)
    for so in (2, 8, 16):
        lhs = np.sum(oracle.first_derivative(g, so, axis, f, kind="forward") * q)
        rhs = -np.sum(f * oracle.first_derivative(g, so, axis, q, kind="backward"))
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)
        # and the central derivative is antisymmetric on its own
        c1 = np.sum(oracle.first_derivative(g, so, axis, f) * q)
        c2 = -np.sum(f * oracle.first_derivative(g, so, axis, q))
        assert abs(c1 - c2) <= 1e-12 * (abs(c1) + 1.0)


def test_staggered_tti_plane_wave_symbols():
    """Constant theta, phi on a periodic grid, staggered reading:
    Hz cos(k.x) = -|sum_j n_j s_j e^{i theta_j/2}|^2 cos(k.x) and
    L cos(k.x) = -|s|^2 cos(k.x), s_d = staggered symbol / h_d."""
    shape = (16, 12, 20)
    h = (0.9, 1.1, 1.0)
    so, r = 8, 4
    th, ph = 0.6, 1.1
    kvec = (2 * math.pi * 3 / (20 * h[0]), 2 * math.pi * 2 / (12 * h[1]),
            2 * math.pi * 4 / (16 * h[2]))
    x, y, z = coords(shape, h)
    q = np.cos(kvec[0] * x + kvec[1] * y + kvec[2] * z)
    thetas = [k * hh for k, hh in zip(kvec, h)]
    s = np.array([fd_exact.staggered_symbol(r, t) / hh for t, hh in zip(thetas, h)])
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    v = sum(n[j] * s[j] * complex(math.cos(thetas[j] / 2), math.sin(thetas[j] / 2))
            for j in range(3))
    hz, lq = oracle.tti_operators(grid(shape, h), so, np.full(shape, th), np.full(shape, ph), q,
                                  periodic=True, deriv="staggered")
    np.testing.assert_allclose(hz, -abs(v) ** 2 * q, atol=1e-11)
    np.testing.assert_allclose(lq, -(s @ s) * q, atol=1e-11)
    # the centred reading gives a different operator on the same wave
    hzc, _ = oracle.tti_operators(grid(shape, h), so, np.full(shape, th), np.full(shape, ph), q,
                                  periodic=True)
    assert np.max(np.abs(hzc - hz)) > 1e-3


def test_staggered_tti_axis_aligned_and_laplacian():
    """theta = 0: Hz = D-z D+z; L = sum_i D-_i D+_i for any angles."""
    shape = (10, 11, 12)
    h = (1.0, 0.8, 1.2)
    g = grid(shape, h)
    q = np.random.default_rng(6).standard_normal(shape)
    so = 8
    Dp = lambda a, f: oracle.first_derivative(g, so, a, f, kind="forward")
    Dm = lambda a, f: oracle.first_derivative(g, so, a, f, kind="backward")
    hz, lq = oracle.tti_operators(g, so, np.zeros(shape), np.full(shape, 0.3), q,
                                  deriv="staggered")
    np.testing.assert_allclose(hz, Dm(2, Dp(2, q)), atol=1e-11)
    np.testing.assert_allclose(lq, sum(Dm(a, Dp(a, q)) for a in range(3)), rtol=1e-12,
                               atol=1e-11)


def test_staggered_tti_operators_are_symmetric_negative():
    """<Hz f, q> = <f, Hz q> <= ... and <Hz f, f> <= 0 with zero ghosts (the
    staggered reading keeps the operator self-adjoint and non-positive)."""
    shape = (8, 9, 10)
    g = grid(shape, (1.0, 1.1, 0.9))
    rng = np.random.default_rng(44)
    th = rng.uniform(0, 1.5, shape)
    ph = rng.uniform(0, 3, shape)
    f = rng.standard_normal(shape)
    q = rng.standard_normal(shape)
    hzf, lf = oracle.tti_operators(g, 8, th, ph, f, deriv="staggered")
    hzq, lq = oracle.tti_operators(g, 8, th, ph, q, deriv="staggered")
    a, b = np.sum(hzf * q), np.sum(f * hzq)
    assert abs(a - b) <= 1e-11 * (abs(a) + 1.0)
    assert np.sum(hzf * f) < 0 and np.sum(lf * f) < 0
    c, d = np.sum(lf * q), np.sum(f * lq)
    assert abs(c - d) <= 1e-11 * (abs(c) + 1.0)


def _tti_case(seed=8, shape=(14, 14, 14), eps=None, delta=None, nt=12):
    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(seed)
    m = (1.0 / rng.uniform(1.5, 2.5, shape) ** 2).astype(np.float32)
    e = np.zeros(shape, np.float32) if eps is None else eps
    d = np.zeros(shape, np.float32) if delta is None else delta
    th = rng.uniform(0, 1.5, shape).astype(np.float32)
    ph = rng.uniform(0, 3, shape).astype(np.float32)
    dt = 1.5
    src = np.array([[[61.3, 72.9, 66.1]]], np.float32)
    wav = workloads.ricker(nt, dt, f0=0.05)[None, :, None].astype(np.float32)
    rec_xyz = np.array([[[40.0, 55.5, 90.2], [100.1, 20.3, 30.7], [70.0, 70.0, 70.0]]],
                       np.float32)
    return grid(shape, h), m, e, d, th, ph, dt, nt, src, wav, rec_xyz


def test_staggered_tti_isotropic_limit_equals_acoustic_with_staggered_laplacian():
    """eps = delta = 0, equal sources: p = r and p obeys m p_tt = sum_i D-_i D+_i p."""
    g, m, e, d, th, ph, dt, nt, src, wav, rec_xyz = _tti_case()
    so = 4
    rec, pf, rf = oracle.tti_forward(g, so, dt, nt, m, e, d, th, ph, src, wav, rec_xyz,
                                     deriv="staggered")
    np.testing.assert_allclose(pf, rf, rtol=1e-12, atol=1e-15)
    Dp = lambda a, f: oracle.first_derivative(g, so, a, f, kind="forward")
    Dm = lambda a, f: oracle.first_derivative(g, so, a, f, kind="backward")
    md = m.astype(np.float64)
    shape = m.shape
    u, um = np.zeros(shape), np.zeros(shape)
    recs = []
    for n in range(nt - 1):
        lap = sum(Dm(a, Dp(a, u)) for a in range(3))
        un = 2 * u - um + dt ** 2 * lap / md
        un = oracle.inject(g, src[0], [wav[0, n, 0]], dt ** 2 / md, un)
        recs.append(oracle.interpolate(g, rec_xyz[0], u))
        um, u = u, un
    recs.append(oracle.interpolate(g, rec_xyz[0], u))
    np.testing.assert_allclose(pf[0, 0], u, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(rec[0], np.array(recs), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("deriv", ["centred", "staggered"])
def test_mean_receivers_record_half_sum_of_p_and_r(deriv):
    """receiver = "mean": rec[n] = interp((p^n + r^n)/2); checked at the last
    step against the interpolation of the final fields, and equal to the p
    receivers in the isotropic limit (p = r)."""
    shape = (12, 12, 12)
    rng = np.random.default_rng(3)
    eps = rng.uniform(0, 0.3, shape).astype(np.float32)
    delta = np.minimum(rng.uniform(0, 0.2, shape).astype(np.float32), eps)
    g, m, e, d, th, ph, dt, nt, src, wav, rec_xyz = _tti_case(seed=9, shape=shape, eps=eps,
                                                               delta=delta, nt=15)
    src = np.array([[[51.3, 52.9, 56.1]]], np.float32)
    rec_m, pf, rf = oracle.tti_forward(g, 4, dt, nt, m, e, d, th, ph, src, wav, rec_xyz,
                                       deriv=deriv, receiver="mean")
    rec_p, pf2, rf2 = oracle.tti_forward(g, 4, dt, nt, m, e, d, th, ph, src, wav, rec_xyz,
                                         deriv=deriv)
    np.testing.assert_array_equal(pf, pf2)
    last = 0.5 * (oracle.interpolate(g, rec_xyz[0], pf[0, 0]) +
                  oracle.interpolate(g, rec_xyz[0], rf[0, 0]))
    np.testing.assert_allclose(rec_m[0, -1], last, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(rec_p[0, -1], oracle.interpolate(g, rec_xyz[0], pf[0, 0]),
                               rtol=1e-12, atol=1e-15)
    assert np.max(np.abs(rec_m - rec_p)) > 1e-3 * np.max(np.abs(rec_p))
    # isotropic limit: p = r, so both receiver readings coincide
    z = np.zeros(shape, np.float32)
    r1, _, _ = oracle.tti_forward(g, 4, dt, nt, m, z, z, th, ph, src, wav, rec_xyz,
                                  deriv=deriv, receiver="mean")
    r2, _, _ = oracle.tti_forward(g, 4, dt, nt, m, z, z, th, ph, src, wav, rec_xyz, deriv=deriv)
    np.testing.assert_allclose(r1, r2, rtol=1e-12, atol=1e-15)


def test_staggered_tti_bounded_when_eps_ge_delta():
    shape = (12, 12, 12)
    h = (10.0, 10.0, 10.0)
    g = grid(shape, h)
    rng = np.random.default_rng(12)
    m = np.full(shape, 1.0 / 2.0 ** 2, np.float32)
    th = rng.uniform(0, 1.2, shape).astype(np.float32)
    ph = rng.uniform(0, 3, shape).astype(np.float32)
    dt = 0.38 * 10.0 / (2.0 * math.sqrt(1 + 2 * 0.3))
    p0 = rng.standard_normal(shape).astype(np.float32)
    init = np.stack([p0, p0])[None]
    empty = np.zeros((1, 0, 3), np.float32)
    nt = 150

    def run(eps, delta):
        _, pf, rf = oracle.tti_forward(g, 4, dt, nt, m, np.full(shape, eps, np.float32),
                                       np.full(shape, delta, np.float32), th, ph, empty,
                                       np.zeros((1, nt, 0), np.float32), empty, p_init=init,
                                       r_init=init.copy(), deriv="staggered")
        return max(np.max(np.abs(pf)), np.max(np.abs(rf))) / np.max(np.abs(p0))

    assert run(0.3, 0.1) < 20.0
    assert run(0.0, 0.6) > 1e3
