"""Pins of the oracle's reduced-precision storage model (binary16 wavefields
and coefficient; the paper's further work on mixed precision, section
"Further work").

The rounding function is checked against numpy's own float16 conversion (an
independent implementation of the same IEEE rounding), the b form of the
update against the m form of the pinned FP64 model, and the storage model
against facts that follow from its definition: every stored value is a
binary16 value, a run without steps returns the rounded initial state, the
first injection from rest lands exactly where hand arithmetic in numpy's
float16 puts it, and the accumulated storage error stays within the size that
per-step rounding allows.

The TTI FP32 storage model (the yardstick for the device's final TTI fields
over long runs) is pinned the same way: it stores FP32 values only, keeps the
initial state, makes one step equal to the rounded FP64 step where the
coefficients are FP32 values, and reduces to the FP64 model without rounding.
"""
import numpy as np
import pytest

import oracle
import workloads


def as_f16(x):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# ---------------------------------------------------------------- rounding

def test_round_binary16_matches_numpy_on_random_magnitudes():
    rng = np.random.default_rng(11)
    x = rng.standard_normal(20000) * 10.0 ** rng.uniform(-9, 5, 20000)
    np.testing.assert_array_equal(oracle.round_binary16(x), as_f16(x))
    x32 = x.astype(np.float32).astype(np.float64)
    np.testing.assert_array_equal(oracle.round_binary16(x32), as_f16(x32))


def test_round_binary16_ties_go_to_even():
    # midpoints between consecutive binary16 values, normal and subnormal,
    # with even and odd lower neighbours; exact in FP64
    h = np.arange(1, 0x7bff, 7, dtype=np.uint16).view(np.float16).astype(np.float64)
    nxt = (np.arange(1, 0x7bff, 7, dtype=np.uint16) + 1).view(np.float16).astype(np.float64)
    mid = 0.5 * (h + nxt)
    got = oracle.round_binary16(np.concatenate([mid, -mid]))
    np.testing.assert_array_equal(got, as_f16(np.concatenate([mid, -mid])))
    low_even = (np.arange(1, 0x7bff, 7) % 2) == 0
    np.testing.assert_array_equal(got[:mid.size], np.where(low_even, h, nxt))


def test_round_binary16_special_values():
    vals = np.array([0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e6, -70000.0, 2.0 ** -24,
                     2.0 ** -25, 2.0 ** -25 * 1.0000001, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25,
                     1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11])
    got = oracle.round_binary16(vals)
    np.testing.assert_array_equal(got, as_f16(vals))
    assert np.signbit(got[1]) and got[1] == 0.0
    assert got[3] == 65504.0 and np.isinf(got[4]) and np.isinf(got[5]) and got[6] < 0
    assert got[8] == 0.0 and got[9] == 2.0 ** -24          # tie to even zero / above the tie
    assert got[12] == 1.0 and got[13] == 1.0 + 2.0 ** -9   # ties to even mantissa
    assert np.isnan(oracle.round_binary16(np.array([np.nan])))[0]


# ---------------------------------------------------------------- model

def _problem(so=8, nt=40, n=32, h=10.0, with_init=True, seed=5):
    shape = (n, n, n)
    v = workloads.smooth_random(shape, seed, 3.0, 1.5, 3.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 6, (h, h, h), 3.0)
    dt = workloads.cfl_dt((h, h, h), 3.0)
    ext = (n - 1) * h
    src = np.array([[[0.43 * ext, 0.51 * ext, 0.47 * ext]]], dtype=np.float32)
    xs = np.linspace(0.1 * ext, 0.9 * ext, 24)
    rec = np.stack([xs, np.full(24, 0.37 * ext), np.full(24, 0.3 * ext)], -1)[None]
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None]
    u0 = workloads.random_wavefields(shape, seed + 1, nshots=1) if with_init else None
    g = oracle.make_grid(shape, (h, h, h))
    return g, so, dt, nt, m, src, wav.astype(np.float32), rec.astype(np.float32), damp, u0


def test_exact_storage_equals_the_m_form_model():
    """The b form u + (1 - b d/dt)(u - u-) + b lap u is algebraically the
    damped leapfrog update: without rounding it reproduces the pinned model."""
    g, so, dt, nt, m, src, wav, rec, damp, u0 = _problem()
    r1, u1 = oracle.acoustic_forward(g, so, dt, nt, m, src, wav, rec, damp=damp, u_init=u0)
    r2, u2 = oracle.acoustic_forward_storage(g, so, dt, nt, m, src, wav, rec, damp=damp,
                                             u_init=u0, storage="exact")
    assert rel(u2, u1) < 1e-12
    assert rel(r2, r1) < 1e-12


def test_f16_storage_holds_only_binary16_values():
    g, so, dt, nt, m, src, wav, rec, damp, u0 = _problem(nt=12)
    r, u = oracle.acoustic_forward_storage(g, so, dt, nt, m, src, wav, rec, damp=damp,
                                           u_init=u0, storage="f16")
    np.testing.assert_array_equal(as_f16(u), u)
    assert np.count_nonzero(u) > 0.9 * u.size
    # receivers interpolate stored values: linear in the stored field
    assert np.all(np.isfinite(r))


def test_f16_no_step_returns_the_rounded_initial_state():
    g, so, dt, nt, m, src, wav, rec, damp, u0 = _problem(nt=1)
    _, u = oracle.acoustic_forward_storage(g, so, dt, 1, m, src, wav[:, :1], rec, damp=damp,
                                           u_init=u0, storage="f16")
    np.testing.assert_array_equal(u[0], as_f16(u0[0]))


def test_f16_first_injection_from_rest_is_hand_rounded():
    """From rest, u^1 holds only the injection: at each corner the stored
    value is f16(f32(w_c b16 q)) with b16 = f16(f32(dt^2/(m + damp dt/2)))."""
    g, so, dt, _, m, src, wav, rec, damp, _ = _problem(nt=2, with_init=False)
    wav = np.zeros((1, 2, 1), np.float32)
    wav[0, 0, 0] = 2.75
    _, u = oracle.acoustic_forward_storage(g, so, dt, 2, m, src, wav, rec, damp=damp,
                                           storage="f16")
    nz, ny, nx = m.shape
    h = g.hx
    s = src[0, 0].astype(np.float64) / h
    i1 = np.floor(s).astype(int)
    fr = s - i1
    expect = np.zeros(m.shape)
    for c in range(8):
        ix, iy, iz = i1[0] + (c & 1), i1[1] + ((c >> 1) & 1), i1[2] + ((c >> 2) & 1)
        wc = ((fr[0] if c & 1 else 1 - fr[0]) * (fr[1] if c & 2 else 1 - fr[1]) *
              (fr[2] if c & 4 else 1 - fr[2]))
        d = damp[ix] + damp[nx + iy] + damp[nx + ny + iz]
        b = dt * dt / (float(m[iz, iy, ix]) + float(d) * dt / 2)
        b16 = float(np.float16(np.float32(b)))
        expect[iz, iy, ix] = float(np.float16(np.float32(wc * b16 * 2.75)))
    np.testing.assert_array_equal(u[0, 0], expect)
    assert np.all(u[0, 1] == 0)


def test_f16_storage_error_is_the_size_rounding_allows():
    """Against the unrounded model the stored run differs by the accumulated
    rounding noise: above one rounding (2^-12 relative) and below the bound
    for nt steps of independent per-step roundings amplified by at most
    1/(omega dt) at the wavelet's peak frequency."""
    g, so, dt, nt, m, src, wav, rec, damp, _ = _problem(nt=150, with_init=False)
    r0, u0 = oracle.acoustic_forward_storage(g, so, dt, nt, m, src, wav, rec, damp=damp,
                                             storage="exact")
    r1, u1 = oracle.acoustic_forward_storage(g, so, dt, nt, m, src, wav, rec, damp=damp,
                                             storage="f16")
    e = rel(u1[0, 0], u0[0, 0])
    omega_dt = 2 * np.pi * 0.03 * dt
    bound = np.sqrt(nt) * 2.0 ** -12 / omega_dt
    assert 2.0 ** -12 < e < bound, (e, bound)
    assert rel(r1, r0) < bound


def test_f16_step_is_the_stored_step_with_binary16_coefficient():
    """One step of the f16 model equals one step with only b in binary16,
    rounded through FP32 to binary16 (the two modes share everything else)."""
    g, so, dt, _, m, src, wav, rec, damp, u0 = _problem(nt=2)
    u0 = as_f16(u0).astype(np.float32)
    _, uf = oracle.acoustic_forward_storage(g, so, dt, 2, m, src, wav[:, :2], rec, damp=damp,
                                            u_init=u0, storage="f16")
    _, uc = oracle.acoustic_forward_storage(g, so, dt, 2, m, src, wav[:, :2] * 0, rec,
                                            damp=damp, u_init=u0, storage="f16_coef")
    _, uz = oracle.acoustic_forward_storage(g, so, dt, 2, m, src, wav[:, :2] * 0, rec,
                                            damp=damp, u_init=u0, storage="f16")
    np.testing.assert_array_equal(uz[0, 0], as_f16(uc[0, 0].astype(np.float32)))
    np.testing.assert_array_equal(uz[0, 1], uc[0, 1])
    assert rel(uf[0, 0], uz[0, 0]) > 0  # the source shows with a nonzero wavelet


# ---------------------------------------------------------------- TTI FP32 storage model

def _tti_case(n=16, nt=3, seed=4, eps_zero=False):
    shape = (n, n, n)
    h = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(seed)
    eps = np.zeros(shape) if eps_zero else rng.uniform(0.0, 0.3, shape)
    delta = np.zeros(shape) if eps_zero else np.minimum(rng.uniform(0.0, 0.2, shape), eps)
    theta = rng.uniform(0.0, np.pi / 4, shape)
    phi = rng.uniform(0.0, np.pi / 4, shape)
    m = workloads.slowness_squared(rng.uniform(1.5, 2.5, shape))
    dt = 0.5 * workloads.cfl_dt(h, 2.5, eps_max=0.3)
    c = (n / 2 - 0.3) * h[0]
    src = np.array([[[c, c, c]]], np.float32)
    rec = np.array([[[c, c - 10.0, c + 15.0], [20.0, 30.0, 40.0]]], np.float32)
    wav = rng.standard_normal((1, nt, 1)).astype(np.float32)
    p0 = (1e-2 * rng.standard_normal((1, 2) + shape)).astype(np.float32)
    r0 = (1e-2 * rng.standard_normal((1, 2) + shape)).astype(np.float32)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    og = oracle.make_grid(shape, h)
    args = (og, 8, dt, nt, m, f32(eps), f32(delta), f32(theta), f32(phi), src, wav, rec)
    return args, p0, r0


def test_tti_f32_storage_stores_fp32_values_and_keeps_the_initial_state():
    """Every value the FP32 storage model stores is an FP32 value, and a run
    without steps returns the initial state (already FP32) unchanged."""
    args, p0, r0 = _tti_case(nt=4)
    _, p, r = oracle.tti_forward(*args, p_init=p0, r_init=r0, storage="f32")
    for f in (p, r):
        np.testing.assert_array_equal(f, f.astype(np.float32).astype(np.float64))
    args1 = args[:3] + (1,) + args[4:10] + (np.zeros((1, 1, 1), np.float32),) + args[11:]
    _, p1, r1 = oracle.tti_forward(*args1, p_init=p0, r_init=r0, storage="f32")
    np.testing.assert_array_equal(p1, p0)
    np.testing.assert_array_equal(r1, r0)


def test_tti_f32_storage_one_step_is_the_rounded_exact_step():
    """With eps = delta = 0 the coefficients a = s = 1 are FP32 values, so one
    step of the storage model is the FP64 step (injection included) rounded
    once to FP32, and the level below it is the initial state."""
    args, p0, r0 = _tti_case(nt=2, eps_zero=True)
    _, pe, re_ = oracle.tti_forward(*args, p_init=p0, r_init=r0)
    _, pm, rm = oracle.tti_forward(*args, p_init=p0, r_init=r0, storage="f32")
    np.testing.assert_array_equal(pm[0, 0], pe[0, 0].astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(rm[0, 0], re_[0, 0].astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(pm[0, 1], p0[0, 0])
    assert np.any(pm[0, 0] != pe[0, 0])  # the rounding did something


def test_tti_f32_storage_rounds_the_coefficients():
    """With eps and delta whose a = 1 + 2 eps and s = sqrt(1 + 2 delta) are
    not FP32 values, one step of the storage model differs from the rounded
    exact step (the coefficients are rounded before they are used), but by no
    more than FP32 rounding of the coefficients can explain (relative 1e-6),
    and the model without rounding is the FP64 model bit for bit."""
    args, p0, r0 = _tti_case(nt=2)
    _, pe, _ = oracle.tti_forward(*args, p_init=p0, r_init=r0)
    _, pm, _ = oracle.tti_forward(*args, p_init=p0, r_init=r0, storage="f32")
    rounded = pe[0, 0].astype(np.float32).astype(np.float64)
    assert np.any(pm[0, 0] != rounded)
    assert rel(pm[0, 0], pe[0, 0]) < 1e-6
    _, px, _ = oracle.tti_forward(*args, p_init=p0, r_init=r0, storage="exact")
    np.testing.assert_array_equal(px, pe)
