"""Pins of the oracle's adjoint and gradient: the dot-product (adjoint) test
and the Taylor test against finite differences of the oracle's own forward
map -- both independent of how the adjoint was derived."""
import numpy as np
import pytest

import oracle
import workloads


def small_problem(so=4, nt=30, nshots=2, seed=0, shape=(14, 12, 16), nbl=3):
    h = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(seed)
    v = workloads.smooth_random(shape, seed + 1, 2.0, 1.5, 2.5)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, nbl, h, 2.5)
    dt = workloads.cfl_dt(h, 2.5)
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    src = (rng.uniform(0.2, 0.8, (nshots, 2, 3)) * ext).astype(np.float32)
    rec = (rng.uniform(0.05, 0.95, (nshots, 7, 3)) * ext).astype(np.float32)
    wav = np.stack([workloads.ricker(nt, dt, f0=0.03)] * 2, -1)[None].repeat(nshots, 0)
    g = oracle.make_grid(shape, h)
    return g, so, dt, nt, m, damp, src, wav.astype(np.float32), rec


@pytest.mark.parametrize("so", [2, 4, 8])
def test_adjoint_dot_product(so):
    g, so, dt, nt, m, damp, src, wav, rec = small_problem(so=so)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(wav.shape).astype(np.float32)
    dd = rng.standard_normal((src.shape[0], nt, rec.shape[1]))
    d, _ = oracle.acoustic_forward(g, so, dt, nt, m, src, q, rec, damp=damp)
    qa = oracle.acoustic_adjoint(g, so, dt, nt, m, src, rec, dd, damp=damp)
    lhs = np.vdot(d, dd)
    rhs = np.vdot(q.astype(np.float64), qa)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-30) + 1e-14 * np.linalg.norm(d) * np.linalg.norm(dd)
    assert abs(lhs) > 0
    # the last source sample never reaches a receiver
    assert np.all(qa[:, -1] == 0)


def _objective(g, so, dt, nt, m, damp, src, wav, rec, dobs):
    d, _ = oracle.acoustic_forward(g, so, dt, nt, m, src, wav, rec, damp=damp)
    return 0.5 * float(np.sum((d - dobs) ** 2)), d


@pytest.mark.parametrize("so", [4, 8])
def test_gradient_taylor(so):
    """J(m + h dm) - J(m) - <g, dm_h> = O(h^2) (second order), while the plain
    difference J(m + h dm) - J(m) is O(h) (first order); dm_h is the actual
    FP32-rounded perturbation."""
    g, so, dt, nt, m, damp, src, wav, rec = small_problem(so=so, nt=40)
    m_true = m
    m0 = workloads.slowness_squared(1.0 / np.sqrt(m_true.astype(np.float64)) * 1.03)
    dobs, _ = oracle.acoustic_forward(g, so, dt, nt, m_true, src, wav, rec, damp=damp)
    J0, d0 = _objective(g, so, dt, nt, m0, damp, src, wav, rec, dobs)
    grad = oracle.acoustic_gradient(g, so, dt, nt, m0, src, wav, rec, d0 - dobs, damp=damp)
    dm = workloads.smooth_random(m0.shape, 9, 2.0, -1.0, 1.0) * float(np.mean(m0))
    r1, r2 = [], []
    for h in (4e-3, 2e-3, 1e-3):
        mp = (m0.astype(np.float64) + h * dm).astype(np.float32)
        dmh = mp.astype(np.float64) - m0.astype(np.float64)
        Jp, _ = _objective(g, so, dt, nt, mp, damp, src, wav, rec, dobs)
        r1.append(abs(Jp - J0))
        r2.append(abs(Jp - J0 - np.vdot(grad, dmh)))
    o1 = [np.log2(r1[i] / r1[i + 1]) for i in range(2)]
    o2 = [np.log2(r2[i] / r2[i + 1]) for i in range(2)]
    assert all(abs(o - 1) < 0.15 for o in o1), (r1, o1)
    assert all(abs(o - 2) < 0.3 for o in o2), (r2, o2)


def test_gradient_is_linear_in_residual_and_sums_shots():
    g, so, dt, nt, m, damp, src, wav, rec = small_problem(so=4, nt=20)
    rng = np.random.default_rng(5)
    dd = rng.standard_normal((2, nt, rec.shape[1]))
    g12 = oracle.acoustic_gradient(g, so, dt, nt, m, src, wav, rec, dd, damp=damp)
    g1 = oracle.acoustic_gradient(g, so, dt, nt, m, src[:1], wav[:1], rec[:1], dd[:1], damp=damp)
    g2 = oracle.acoustic_gradient(g, so, dt, nt, m, src[1:], wav[1:], rec[1:], dd[1:], damp=damp)
    np.testing.assert_allclose(g12, g1 + g2, rtol=1e-12, atol=1e-12 * np.abs(g12).max())
    g3 = oracle.acoustic_gradient(g, so, dt, nt, m, src, wav, rec, 3.0 * dd, damp=damp)
    np.testing.assert_allclose(g3, 3.0 * g12, rtol=1e-12, atol=1e-12 * np.abs(g12).max())
