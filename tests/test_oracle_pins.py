"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper prints (Listing fd-1,
fd-3, finject), a closed form (Taylor moment conditions solved exactly, the
discrete dispersion relation, the stencil symbol), an invariant (discrete
energy, operator symmetry, adjointness) or a special case, chosen so that a
dropped term, a wrong sign, a transposed axis or a wrong coefficient
placement fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import fd_exact
import workloads

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def grid(shape, h=(1.0, 1.0, 1.0), o=(0.0, 0.0, 0.0)):
    return oracle.make_grid(shape, h, o)


def coords(shape, h, o=(0.0, 0.0, 0.0)):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) * h[2] + o[2], np.arange(ny) * h[1] + o[1],
                          np.arange(nx) * h[0] + o[0], indexing="ij")
    return x, y, z


# ----------------------------------------------------------------- FD weights

@pytest.mark.parametrize("r", range(1, 9))
def test_weights_match_exact_moment_solution(r):
    w, c = oracle.fd_weights(r)
    we = [float(v) for v in fd_exact.second_derivative_weights(r)]
    ce = [float(v) for v in fd_exact.first_derivative_weights(r)]
    np.testing.assert_allclose(w, we, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(c, ce, rtol=1e-13, atol=1e-15)


def test_weights_radius1_are_listing_fd1():
    g = GOLDEN["listing_fd1"]
    w, c = oracle.fd_weights(1)
    assert w[0] == g["u_dt2_weights_times_dt2"]["0"]
    assert w[1] == g["u_dt2_weights_times_dt2"]["1"] == g["u_dt2_weights_times_dt2"]["-1"]
    assert c[1] == g["u_dx_weights_times_h"]["1"] == -g["u_dx_weights_times_h"]["-1"]


def test_weights_radius2_known_values():
    w, c = oracle.fd_weights(2)
    np.testing.assert_allclose(w, [-5 / 2, 4 / 3, -1 / 12], rtol=1e-15)
    np.testing.assert_allclose(c, [0, 2 / 3, -1 / 12], rtol=1e-15)


@pytest.mark.parametrize("r", [1, 2, 4, 6, 8])
def test_weights_polynomial_exactness(r):
    """Second derivative exact on x^p for p <= 2r+1, wrong at p = 2r+2; first
    derivative exact for p <= 2r, wrong at p = 2r+1 (evaluated at x0 = 0.37)."""
    w, c = oracle.fd_weights(r)
    x0 = 0.37
    ks = np.arange(1, r + 1)
    for p in range(0, 2 * r + 3):
        f = lambda x: x ** p
        d2 = w[0] * f(x0) + np.sum(w[1:] * (f(x0 + ks) + f(x0 - ks)))
        d2_exact = p * (p - 1) * x0 ** (p - 2) if p >= 2 else 0.0
        if p <= 2 * r + 1:
            assert abs(d2 - d2_exact) <= 1e-9 * max(1.0, abs(d2_exact)) * (r + 1) ** p / 10
        if p == 2 * r + 2:
            assert abs(d2 - d2_exact) > 1e-6 * abs(d2_exact)
        d1 = np.sum(c[1:] * (f(x0 + ks) - f(x0 - ks)))
        d1_exact = p * x0 ** (p - 1) if p >= 1 else 0.0
        if p <= 2 * r:
            assert abs(d1 - d1_exact) <= 1e-9 * max(1.0, abs(d1_exact)) * (r + 1) ** p / 10
        if p == 2 * r + 1:
            assert abs(d1 - d1_exact) > 1e-6 * abs(d1_exact)


def test_stencil_point_count_so8_is_25():
    """The so=8 compact Laplacian touches 25 points (figure 'folds' caption)."""
    g = grid((17, 17, 17))
    u = np.zeros((17, 17, 17))
    u[8, 8, 8] = 1.0
    lap = oracle.laplacian(g, GOLDEN["stencil_points"]["space_order"], u)
    assert np.count_nonzero(lap) == GOLDEN["stencil_points"]["points"]


# ----------------------------------------------------------------- spatial operators

@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_laplacian_exact_on_polynomials_interior(so):
    r = so // 2
    h = (0.5, 0.25, 0.4)
    shape = (2 * r + 3, 2 * r + 4, 2 * r + 5)
    x, y, z = coords(shape, h, (-1.0, 0.3, -0.7))
    a, b, cc = min(so + 1, 5), min(so + 1, 4), min(so + 1, 3)
    u = x ** a * y ** b + z ** cc * x + 2.0 * y ** 2 * z
    lap_exact = (a * (a - 1) * x ** (a - 2) * y ** b + b * (b - 1) * x ** a * y ** (b - 2)
                 + cc * (cc - 1) * z ** (cc - 2) * x + 4.0 * z)
    lap = oracle.laplacian(grid(shape, h, (-1.0, 0.3, -0.7)), so, u)
    inner = (slice(r, -r), slice(r, -r), slice(r, -r))
    np.testing.assert_allclose(lap[inner], lap_exact[inner], rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("so,ns", [(4, [16, 24, 36]), (8, [12, 16, 20]), (12, [10, 12, 14]),
                                   (16, [8, 10, 12])])
def test_laplacian_convergence_order(so, ns):
    """Error on a periodic smooth field decreases as h^so (observed order)."""
    L = 2 * math.pi
    errs = []
    for n in ns:
        h = L / n
        x, y, z = coords((n, n, n), (h, h, h))
        u = np.sin(x) * np.sin(y) * np.cos(z)
        lap = oracle.laplacian(grid((n, n, n), (h, h, h)), so, u, periodic=True)
        errs.append(np.max(np.abs(lap + 3.0 * u)))
    orders = [math.log(errs[i] / errs[i + 1]) / math.log(ns[i + 1] / ns[i]) for i in range(2)]
    assert all(abs(o - so) < 1.0 for o in orders), (errs, orders)


@pytest.mark.parametrize("so", [4, 12])
def test_laplacian_symbol_on_periodic_plane_wave(so):
    """lap cos(k.x) = -sum_d sigma(k_d h_d)/h_d^2 cos(k.x): exact stencil symbol
    from independently derived weights; distinct k and h per axis."""
    r = so // 2
    shape = (20, 16, 24)  # nz, ny, nx
    h = (0.7, 1.1, 0.9)
    kx, ky, kz = 2 * math.pi * 3 / (24 * h[0]), 2 * math.pi * 2 / (16 * h[1]), 2 * math.pi * 5 / (20 * h[2])
    x, y, z = coords(shape, h)
    u = np.cos(kx * x + ky * y + kz * z)
    lam = sum(fd_exact.second_symbol(r, k * hh) / hh ** 2 for k, hh in ((kx, h[0]), (ky, h[1]), (kz, h[2])))
    lap = oracle.laplacian(grid(shape, h), so, u, periodic=True)
    np.testing.assert_allclose(lap, -lam * u, atol=1e-11 * lam)


def test_laplacian_dirichlet_is_symmetric():
    rng = np.random.default_rng(11)
    shape = (9, 11, 13)
    g = grid(shape, (1.0, 0.8, 1.3))
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    for so in (4, 16):
        a = np.vdot(v, oracle.laplacian(g, so, u))
        b = np.vdot(oracle.laplacian(g, so, v), u)
        assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_first_derivative_exact_and_antisymmetric(axis):
    so, r = 8, 4
    h = (0.5, 0.7, 0.3)
    shape = (13, 12, 11)
    x, y, z = coords(shape, h, (0.2, -0.4, 0.1))
    X = (x, y, z)[axis]
    f = X ** 5 + 3 * X ** 2 * (y + 1.0) * (z - 2.0) * (x + 0.5)
    g = grid(shape, h, (0.2, -0.4, 0.1))
    d = oracle.first_derivative(g, so, axis, f)
    # exact derivative along `axis` of f
    eps = [x, y, z]
    if axis == 0:
        exact = 5 * x ** 4 + 3 * (2 * x * (x + 0.5) + x ** 2) * (y + 1.0) * (z - 2.0)
    elif axis == 1:
        exact = 5 * y ** 4 + 3 * (2 * y * (y + 1.0) + y ** 2) * (z - 2.0) * (x + 0.5)
    else:
        exact = 5 * z ** 4 + 3 * (2 * z * (z - 2.0) + z ** 2) * (y + 1.0) * (x + 0.5)
    del eps
    inner = (slice(r, -r), slice(r, -r), slice(r, -r))
    np.testing.assert_allclose(d[inner], exact[inner], rtol=1e-9, atol=1e-9)
    rng = np.random.default_rng(axis)
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    a = np.vdot(v, oracle.first_derivative(g, so, axis, u))
    b = np.vdot(oracle.first_derivative(g, so, axis, v), u)
    assert abs(a + b) < 1e-12 * (abs(a) + 1.0)


# ----------------------------------------------------------------- leapfrog in time

def test_one_dimensional_step_is_listing_fd3():
    """so = 2, a 1-D line (periodic in y and z with one point, so their second
    differences vanish): the oracle step equals Listing fd-3 term by term."""
    gv = GOLDEN["listing_fd3"]
    n, h, dt = 12, 0.5, 0.1
    rng = np.random.default_rng(3)
    u = rng.standard_normal((1, 1, n))
    up = rng.standard_normal((1, 1, n))
    m = rng.uniform(0.5, 2.0, (1, 1, n))
    g = grid((1, 1, n), (h, 1.0, 1.0))
    out = oracle.acoustic_step(g, 2, dt, m, u, up, periodic=True)
    uu, uq, mm = u[0, 0], up[0, 0], m[0, 0]
    k = dt ** 2 / (h ** 2 * mm)
    c = gv["coeff_dt2_over_h2m"]
    exp = (c["x"] * k * uu + c["x-h"] * k * np.roll(uu, 1) + c["x+h"] * k * np.roll(uu, -1)
           + gv["coeff_u_t"] * uu + gv["coeff_u_tm1"] * uq)
    np.testing.assert_allclose(out[0, 0], exp, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("so", [4, 16])
def test_plane_wave_follows_discrete_dispersion(so):
    """Periodic plane wave cos(k.x - w n dt) with (2/dt)^2 sin^2(w dt/2) =
    v^2 sum_d sigma(k_d h_d)/h_d^2 is reproduced to rounding after 60 steps."""
    r = so // 2
    shape = (12, 10, 14)
    h = (10.0, 12.0, 9.0)
    v = 2.0
    kx, ky, kz = 2 * math.pi * 2 / (14 * h[0]), 2 * math.pi * 1 / (10 * h[1]), 2 * math.pi * 3 / (12 * h[2])
    lam = sum(fd_exact.second_symbol(r, k * hh) / hh ** 2 for k, hh in ((kx, h[0]), (ky, h[1]), (kz, h[2])))
    dt = 0.3 * min(h) / v
    w = 2.0 / dt * math.asin(0.5 * dt * v * math.sqrt(lam))
    x, y, z = coords(shape, h)
    ph = kx * x + ky * y + kz * z
    u_init = np.stack([np.cos(ph), np.cos(ph + w * dt)])[None].astype(np.float32)
    # FP32-rounded initial data: compare against the exact evolution of those data
    # by running the closed form on both components (linear in the initial data).
    m = np.full(shape, 1.0 / v ** 2, dtype=np.float32)
    nt = 61
    g = grid(shape, h)
    empty = np.zeros((1, 0, 3), np.float32)
    _, uf = oracle.acoustic_forward(g, so, dt, nt, m, empty, np.zeros((1, nt, 0), np.float32),
                                    empty, u_init=u_init, periodic=True)
    # m was rounded to FP32 too: use the dispersion of the rounded m
    v32 = 1.0 / math.sqrt(float(m.flat[0]))
    w32 = 2.0 / dt * math.asin(0.5 * dt * v32 * math.sqrt(lam))
    # exact solution from the two FP32 initial levels: a cos + b sin split is not
    # needed because both levels are (rounded) samples of the same wave; the
    # rounding error (1e-7) propagates linearly and boundedly.
    exact = np.cos(ph - w32 * (nt - 1) * dt)
    assert abs(w32 - w) < 1e-6 * w
    np.testing.assert_allclose(uf[0, 0], exact, atol=5e-5)
    # With FP64 data the same closed form holds to 1e-10 (stepping manually)
    u0, um = np.cos(ph), np.cos(ph + w * dt)
    mm = np.full(shape, 1.0 / v ** 2)
    for _ in range(nt - 1):
        u0, um = oracle.acoustic_step(g, so, dt, mm, u0, um, periodic=True), u0
    np.testing.assert_allclose(u0, np.cos(ph - w * (nt - 1) * dt), atol=1e-10)


def _energy(g, so, dt, m, un1, un):
    """E^{n+1/2} = 1/2 ||(u^{n+1}-u^n)/dt||_m^2 - 1/2 <u^{n+1}, L u^n>."""
    lap = oracle.laplacian(g, so, un)
    return 0.5 * np.sum(m * ((un1 - un) / dt) ** 2) - 0.5 * np.vdot(un1, lap)


def _cfl_bound(so, h, vmax):
    """Exact leapfrog bound dt <= 2 / (vmax sqrt(sum_d sigma(pi)/h_d^2))."""
    s = fd_exact.second_symbol(so // 2, math.pi)
    return 2.0 / (vmax * math.sqrt(sum(s / hh ** 2 for hh in h)))


@pytest.mark.parametrize("so", [4, 8])
def test_energy_conserved_undamped_dirichlet(so):
    shape = (14, 13, 12)
    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(5)
    m = 1.0 / rng.uniform(1.5, 3.0, shape) ** 2
    vmax = float(np.max(1.0 / np.sqrt(m)))
    dt = 0.9 * _cfl_bound(so, h, vmax)
    g = grid(shape, h)
    u = workloads.smooth_random(shape, 3, 1.5, -1, 1)
    um = workloads.smooth_random(shape, 4, 1.5, -1, 1)
    es = []
    for _ in range(40):
        un = oracle.acoustic_step(g, so, dt, m, u, um)
        es.append(_energy(g, so, dt, m, un, u))
        um, u = u, un
    es = np.array(es)
    assert es.min() > 0
    assert np.max(np.abs(es - es[0])) < 1e-11 * es[0]


def test_energy_non_increasing_with_damping():
    so = 4
    shape = (16, 16, 16)
    h = (10.0, 10.0, 10.0)
    m = np.full(shape, 1.0 / 2.0 ** 2)
    dt = 0.8 * _cfl_bound(so, h, 2.0)
    damp = workloads.damping_profile(shape, 5, h, 2.0).astype(np.float64)
    g = grid(shape, h)
    u = workloads.smooth_random(shape, 8, 2.0, -1, 1)
    um = u.copy()
    es = []
    for _ in range(60):
        un = oracle.acoustic_step(g, so, dt, m, u, um, damp=damp)
        es.append(_energy(g, so, dt, m, un, u))
        um, u = u, un
    d = np.diff(es)
    assert np.all(d <= 1e-12 * es[0])
    assert es[-1] < 0.9 * es[0]


def test_unstable_above_cfl_bound():
    so = 4
    shape = (12, 12, 12)
    h = (10.0, 10.0, 10.0)
    m = np.full(shape, 1.0 / 3.0 ** 2)
    g = grid(shape, h)
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal(shape)
    growth = {}
    for fac in (0.98, 1.05):
        dt = fac * _cfl_bound(so, h, 3.0)
        u, um = u0.copy(), u0.copy()
        for _ in range(200):
            u, um = oracle.acoustic_step(g, so, dt, m, u, um), u
        growth[fac] = np.max(np.abs(u)) / np.max(np.abs(u0))
    assert growth[0.98] < 10.0
    assert growth[1.05] > 1e3


def test_cfl_rule_matches_paper_step_counts():
    """dt = 0.38 h / v_max reproduces the paper's step counts to within 1%
    (v_max = 2.5 km/s; TTI with eps_max = 0.3)."""
    g = GOLDEN["test_case_setup"]
    h, T = g["h_m"], g["t_end_ms"]
    n_iso = workloads.steps_for(T, workloads.cfl_dt((h, h, h), 2.5))
    n_tti = workloads.steps_for(T, workloads.cfl_dt((h, h, h), 2.5, eps_max=0.3))
    assert abs(n_iso - g["steps_isotropic"]) <= 0.01 * g["steps_isotropic"]
    assert abs(n_tti - g["steps_tti"]) <= 0.01 * g["steps_tti"]
    # and 0.38 sits below the exact compact-stencil bound for every space order
    for so in (4, 8, 12, 16):
        assert workloads.CFL_FACTOR * 20.0 / 2.5 < _cfl_bound(so, (20.0,) * 3, 2.5)


def test_manufactured_solution_second_order_in_time():
    """u = sin(x) sin(y) sin(z) cos(w t) with forcing f = m u_tt - lap u on a
    periodic box, so = 16 (spatial error negligible): error ~ dt^2."""
    so, n = 16, 16
    L = 2 * math.pi
    h = L / n
    x, y, z = coords((n, n, n), (h, h, h))
    S = np.sin(x) * np.sin(y) * np.sin(z)
    m = np.full((n, n, n), 0.5)
    w = 1.7
    T = 2.0
    g = grid((n, n, n), (h, h, h))
    errs = []
    for nsteps in (40, 80):
        dt = T / nsteps
        f = lambda t: (-0.5 * w ** 2 + 3.0) * S * math.cos(w * t)
        u, um = S.copy(), S * math.cos(-w * dt)
        for k in range(nsteps):
            un = oracle.acoustic_step(g, so, dt, m, u, um, periodic=True)
            un += dt ** 2 * f(k * dt) / m
            um, u = u, un
        errs.append(np.max(np.abs(u - S * math.cos(w * T))))
    order = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert abs(order - 2.0) < 0.2, (errs, order)


# ----------------------------------------------------------------- sparse operators

def test_interpolation_reproduces_affine_fields():
    shape = (7, 8, 9)
    h, o = (2.0, 3.0, 1.5), (-5.0, 1.0, 0.5)
    x, y, z = coords(shape, h, o)
    u = 1.25 + 0.5 * x - 2.0 * y + 0.75 * z
    rng = np.random.default_rng(1)
    pts = np.stack([rng.uniform(o[0], o[0] + 8 * h[0], 50), rng.uniform(o[1], o[1] + 7 * h[1], 50),
                    rng.uniform(o[2], o[2] + 6 * h[2], 50)], -1).astype(np.float32)
    pts[0] = [o[0] + 8 * h[0], o[1] + 7 * h[1], o[2] + 6 * h[2]]  # last node in every axis
    pts[1] = [o[0], o[1], o[2]]
    got = oracle.interpolate(grid(shape, h, o), pts, u)
    p = pts.astype(np.float64)
    np.testing.assert_allclose(got, 1.25 + 0.5 * p[:, 0] - 2.0 * p[:, 1] + 0.75 * p[:, 2],
                               rtol=1e-12, atol=1e-12)


def test_injection_is_adjoint_of_interpolation_and_partition_of_unity():
    shape = (6, 7, 8)
    h = (1.0, 2.0, 0.5)
    g = grid(shape, h)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.uniform(0, 7, 20), rng.uniform(0, 12, 20), rng.uniform(0, 2.5, 20)],
                   -1).astype(np.float32)
    u = rng.standard_normal(shape)
    d = rng.standard_normal(20)
    ones = np.ones(shape)
    Pu = oracle.interpolate(g, pts, u)
    PTd = oracle.inject(g, pts, d, ones, np.zeros(shape))
    assert abs(np.dot(Pu, d) - np.vdot(u, PTd)) < 1e-13 * np.sum(np.abs(d)) * np.max(np.abs(u)) * 8
    tot = oracle.inject(g, pts, np.ones(20), ones, np.zeros(shape))
    assert abs(tot.sum() - 20.0) < 1e-12


def test_injection_matches_listing_finject():
    """A point on-node in y and z, off-node in x: the injected values at x1 and
    x1+1 are Listing finject's dt^2 (1-frac) q / m[x1] and dt^2 frac q / m[x1+1]."""
    shape = (4, 4, 10)
    h, o = (2.5, 1.0, 1.0), (-3.0, 0.0, 0.0)
    g = grid(shape, h, o)
    dt, q = 0.7, 1.9
    m = np.random.default_rng(4).uniform(0.2, 0.9, shape)
    xq = np.float32(-3.0 + 4.3 * 2.5)
    pts = np.array([[xq, 2.0, 1.0]], np.float32)
    out = oracle.inject(g, pts, [q], dt ** 2 / m, np.zeros(shape))
    x1 = math.floor((float(xq) - o[0]) / h[0])
    frac = (float(xq) - o[0] - h[0] * x1) / h[0]
    exp = np.zeros(shape)
    exp[1, 2, x1] = dt ** 2 * (1 - frac) * q / m[1, 2, x1]
    exp[1, 2, x1 + 1] = dt ** 2 * frac * q / m[1, 2, x1 + 1]
    np.testing.assert_allclose(out, exp, rtol=1e-12, atol=1e-15)


def test_out_of_grid_point_is_rejected():
    g = grid((4, 4, 4))
    with pytest.raises(oracle.OracleError):
        oracle.interpolate(g, np.array([[3.0001, 1.0, 1.0]], np.float32), np.zeros((4, 4, 4)))
    with pytest.raises(oracle.OracleError):
        oracle.interpolate(g, np.array([[1.0, -0.001, 1.0]], np.float32), np.zeros((4, 4, 4)))


# ----------------------------------------------------------------- forward composition

def _point_problem(nt=30, nshots=1):
    w = workloads.acoustic_small(so=4, nt=nt)
    return w


def test_forward_first_steps_compose_as_scheduled():
    """From rest: u^1 is exactly the injection of src[0]; rec[0] = 0;
    rec[1] = interp(u^1) (stencil, then injection into t+1, receivers at t)."""
    w = workloads.acoustic_small(so=4, nt=2)
    g = oracle.make_grid(w.shape, w.spacing, w.origin)
    wav = np.zeros_like(w.src_wav)
    wav[0, 0, 0] = 3.0
    rec_xyz = np.concatenate([w.rec_xyz, w.src_xyz], axis=1)
    rec, uf = oracle.acoustic_forward(g, w.so, w.dt, 2, w.m, w.src_xyz, wav, rec_xyz, damp=w.damp)
    m = w.m.astype(np.float64)
    u1 = oracle.inject(g, w.src_xyz[0], [3.0], w.dt ** 2 / m, np.zeros(w.shape))
    np.testing.assert_allclose(uf[0, 0], u1, rtol=1e-14, atol=0)
    assert np.all(uf[0, 1] == 0)
    assert np.all(rec[0, 0] == 0)
    np.testing.assert_allclose(rec[0, 1], oracle.interpolate(g, rec_xyz[0], u1), rtol=1e-14)


def test_forward_linear_in_source_and_shots_independent():
    w = workloads.acoustic_small(so=8, nt=25)
    g = oracle.make_grid(w.shape, w.spacing, w.origin)
    rec1, uf1 = oracle.acoustic_forward(g, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                        w.rec_xyz, damp=w.damp)
    src2 = np.concatenate([w.src_xyz, w.src_xyz + np.float32(13.0)], 0)
    wav2 = np.concatenate([w.src_wav, 2.0 * w.src_wav], 0)
    rec2, uf2 = oracle.acoustic_forward(g, w.so, w.dt, w.nt, w.m, src2, wav2,
                                        np.concatenate([w.rec_xyz] * 2, 0), damp=w.damp)
    np.testing.assert_array_equal(rec2[0], rec1[0])
    np.testing.assert_array_equal(uf2[0], uf1[0])
    rec3, _ = oracle.acoustic_forward(g, w.so, w.dt, w.nt, w.m, src2[1:], w.src_wav,
                                      w.rec_xyz, damp=w.damp)
    np.testing.assert_allclose(rec2[1], 2.0 * rec3[0], rtol=1e-12, atol=1e-300)


def test_source_receiver_reciprocity_constant_medium():
    """Injection is the adjoint of interpolation: in a constant medium the
    trace at B from a source at A equals the trace at A from a source at B."""
    shape = (20, 20, 20)
    h = (10.0, 10.0, 10.0)
    g = grid(shape, h)
    m = np.full(shape, np.float32(1 / 2.0 ** 2), dtype=np.float32)
    dt = 0.38 * 10.0 / 2.0
    nt = 40
    A = np.array([[[62.3, 81.7, 95.1]]], np.float32)
    B = np.array([[[121.9, 104.4, 77.2]]], np.float32)
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None].astype(np.float32)
    damp = workloads.damping_profile(shape, 4, h, 2.0)
    rAB, _ = oracle.acoustic_forward(g, 4, dt, nt, m, A, wav, B, damp=damp)
    rBA, _ = oracle.acoustic_forward(g, 4, dt, nt, m, B, wav, A, damp=damp)
    np.testing.assert_allclose(rAB, rBA, rtol=1e-10, atol=1e-12 * np.max(np.abs(rAB)))
    assert np.max(np.abs(rAB)) > 0


# ----------------------------------------------------------------- TTI

def test_tti_axis_aligned_reduces_to_second_first_derivative():
    """theta = 0 -> Hz = Dz Dz; theta = pi/2, phi = 0 -> Dx Dx; phi = pi/2 -> Dy Dy;
    and L = Dx Dx + Dy Dy + Dz Dz for any angles."""
    shape = (10, 11, 12)
    h = (1.0, 0.8, 1.2)
    g = grid(shape, h)
    q = np.random.default_rng(6).standard_normal(shape)
    so = 8
    D = lambda a, f: oracle.first_derivative(g, so, a, f)
    cases = [(0.0, 0.3, 2), (math.pi / 2, 0.0, 0), (math.pi / 2, math.pi / 2, 1)]
    for th, ph, axis in cases:
        hz, lq = oracle.tti_operators(g, so, np.full(shape, th), np.full(shape, ph), q)
        np.testing.assert_allclose(hz, D(axis, D(axis, q)), atol=1e-11)
        np.testing.assert_allclose(lq, sum(D(a, D(a, q)) for a in range(3)), rtol=1e-12, atol=1e-11)


def test_tti_plane_wave_symbols():
    """Constant theta, phi on a periodic grid: Hz cos(k.x) = -(n.s)^2 cos(k.x),
    L cos(k.x) = -|s|^2 cos(k.x), s_d = first-derivative symbol / h_d."""
    shape = (16, 12, 20)
    h = (0.9, 1.1, 1.0)
    so, r = 8, 4
    th, ph = 0.6, 1.1
    kx, ky, kz = (2 * math.pi * 3 / (20 * h[0]), 2 * math.pi * 2 / (12 * h[1]),
                  2 * math.pi * 4 / (16 * h[2]))
    x, y, z = coords(shape, h)
    q = np.cos(kx * x + ky * y + kz * z)
    s = np.array([fd_exact.first_symbol(r, k * hh) / hh for k, hh in ((kx, h[0]), (ky, h[1]), (kz, h[2]))])
    n = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    hz, lq = oracle.tti_operators(grid(shape, h), so, np.full(shape, th), np.full(shape, ph), q,
                                  periodic=True)
    np.testing.assert_allclose(hz, -(n @ s) ** 2 * q, atol=1e-11)
    np.testing.assert_allclose(lq, -(s @ s) * q, atol=1e-11)


def test_tti_one_step_coupling_constant_medium():
    """One TTI step of plane waves in a constant periodic medium matches the
    closed form: P+ = 2P - P- + dt^2/m ((1+2e) X P + sqrt(1+2d) Z R),
    R+ = 2R - R- + dt^2/m (sqrt(1+2d) X P + Z R), X = -(|s|^2-(n.s)^2), Z = -(n.s)^2."""
    shape = (12, 10, 14)
    h = (10.0, 10.0, 10.0)
    so, r = 4, 2
    th, ph, e, d = 0.5, 0.25, 0.25, 0.1
    kx, ky, kz = (2 * math.pi * 2 / (14 * h[0]), 2 * math.pi * 3 / (10 * h[1]),
                  2 * math.pi * 1 / (12 * h[2]))
    x, y, z = coords(shape, h)
    c = np.cos(kx * x + ky * y + kz * z)
    P0, Pm, R0, Rm = 1.0, 0.9, 0.7, 0.8
    f32 = lambda v: np.full(shape, v, np.float32)
    m = f32(1 / 2.0 ** 2)
    eps, dl = f32(e), f32(d)
    thf, phf = f32(th), f32(ph)
    dt = 2.0
    p_init = np.stack([P0 * c, Pm * c])[None].astype(np.float32)
    r_init = np.stack([R0 * c, Rm * c])[None].astype(np.float32)
    empty = np.zeros((1, 0, 3), np.float32)
    _, pf, rf = oracle.tti_forward(grid(shape, h), so, dt, 2, m, eps, dl, thf, phf, empty,
                                   np.zeros((1, 2, 0), np.float32), empty, p_init=p_init,
                                   r_init=r_init, periodic=True)
    s = np.array([fd_exact.first_symbol(r, k * 10.0) / 10.0 for k in (kx, ky, kz)])
    thd, phd = float(thf.flat[0]), float(phf.flat[0])
    n = np.array([math.sin(thd) * math.cos(phd), math.sin(thd) * math.sin(phd), math.cos(thd)])
    X = -(s @ s - (n @ s) ** 2)
    Z = -(n @ s) ** 2
    a = 1 + 2 * float(eps.flat[0])
    sd = math.sqrt(1 + 2 * float(dl.flat[0]))
    mm = float(m.flat[0])
    p_in, r_in = p_init[0].astype(np.float64), r_init[0].astype(np.float64)
    Pexp = 2 * p_in[0] - p_in[1] + dt ** 2 / mm * (a * X * p_in[0] + sd * Z * r_in[0])
    Rexp = 2 * r_in[0] - r_in[1] + dt ** 2 / mm * (sd * X * p_in[0] + Z * r_in[0])
    # the FP32-rounded initial plane waves carry 1e-8 rounding noise that the
    # operator amplifies; a misplaced coefficient changes the result by > 1e-3
    np.testing.assert_allclose(pf[0, 0], Pexp, atol=5e-8)
    np.testing.assert_allclose(rf[0, 0], Rexp, atol=5e-8)
    assert np.max(np.abs(Pexp - Rexp)) > 1e-2


def test_tti_isotropic_limit_equals_acoustic_with_dd_laplacian():
    """eps = delta = 0, equal p and r sources: p obeys m p_tt = (Dx Dx + Dy Dy +
    Dz Dz) p for any theta, phi (built here from the pinned first derivative)."""
    shape = (14, 14, 14)
    h = (10.0, 10.0, 10.0)
    so = 4
    g = grid(shape, h)
    rng = np.random.default_rng(8)
    m = (1.0 / rng.uniform(1.5, 2.5, shape) ** 2).astype(np.float32)
    zero = np.zeros(shape, np.float32)
    th = rng.uniform(0, 1.5, shape).astype(np.float32)
    ph = rng.uniform(0, 3, shape).astype(np.float32)
    dt, nt = 1.5, 12
    src = np.array([[[61.3, 72.9, 66.1]]], np.float32)
    wav = workloads.ricker(nt, dt, f0=0.05)[None, :, None].astype(np.float32)
    rec_xyz = np.array([[[40.0, 55.5, 90.2], [100.1, 20.3, 30.7]]], np.float32)
    rec, pf, rf = oracle.tti_forward(g, so, dt, nt, m, zero, zero, th, ph, src, wav, rec_xyz)
    np.testing.assert_allclose(pf, rf, rtol=1e-12, atol=1e-15)
    # reference: leapfrog with the D o D Laplacian built from pinned operators
    D = lambda a, f: oracle.first_derivative(g, so, a, f)
    md = m.astype(np.float64)
    u, um = np.zeros(shape), np.zeros(shape)
    recs = []
    for n in range(nt - 1):
        lap = sum(D(a, D(a, u)) for a in range(3))
        un = 2 * u - um + dt ** 2 * lap / md
        un = oracle.inject(g, src[0], [wav[0, n, 0]], dt ** 2 / md, un)
        recs.append(oracle.interpolate(g, rec_xyz[0], u))
        um, u = u, un
    recs.append(oracle.interpolate(g, rec_xyz[0], u))
    np.testing.assert_allclose(pf[0, 0], u, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(rec[0], np.array(recs), rtol=1e-11, atol=1e-14)


def _tti_energy_run(eps, delta, nt=150):
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
    _, pf, rf = oracle.tti_forward(g, 4, dt, nt, m, np.full(shape, eps, np.float32),
                                   np.full(shape, delta, np.float32), th, ph, empty,
                                   np.zeros((1, nt, 0), np.float32), empty, p_init=init,
                                   r_init=init.copy())
    return max(np.max(np.abs(pf)), np.max(np.abs(rf))) / np.max(np.abs(p0))


def test_tti_bounded_when_eps_ge_delta_and_grows_otherwise():
    assert _tti_energy_run(0.3, 0.1) < 20.0
    assert _tti_energy_run(0.0, 0.6) > 1e3


def test_reciprocity_inside_damping_layer():
    """With the damped update (m+eta) u+ = dt^2 L u + 2 m u - (m-eta) u- + dt^2 P^T q
    the z-transformed operator is symmetric, so reciprocity also holds for a
    source and a receiver inside the absorbing border (different damping at
    each); any other injection scale there breaks it."""
    shape = (20, 20, 20)
    h = (10.0, 10.0, 10.0)
    g = grid(shape, h)
    m = np.full(shape, np.float32(1 / 2.0 ** 2), dtype=np.float32)
    dt = 0.38 * 10.0 / 2.0
    nt = 40
    damp = workloads.damping_profile(shape, 6, h, 2.0)
    A = np.array([[[22.3, 81.7, 95.1]]], np.float32)   # x inside the border
    B = np.array([[[121.9, 104.4, 11.2]]], np.float32)  # z inside the border
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None].astype(np.float32)
    rAB, _ = oracle.acoustic_forward(g, 4, dt, nt, m, A, wav, B, damp=damp)
    rBA, _ = oracle.acoustic_forward(g, 4, dt, nt, m, B, wav, A, damp=damp)
    np.testing.assert_allclose(rAB, rBA, rtol=1e-10, atol=1e-12 * np.max(np.abs(rAB)))
    assert np.max(np.abs(rAB)) > 0
