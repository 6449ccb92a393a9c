"""Failure handling on the GPU, in forms that fault, trap or hang nothing.

* Divergence: a non-finite or overflowing initial state makes the time loop's
  watchdog (a sampled finiteness check every 16 steps) set the device error
  flag; the stencil launches after it return at once and the call reports
  FD_ERR_DIVERGED without running its whole time budget.
* Allocation failure: FDSWEEP_FAIL_ALLOC=1 makes the library's device
  allocations fail as if the device were full (a fake of the failing call, on
  the host); calls return FD_ERR_OOM and launch nothing.
* Bounded waits: fd_set_wait_limit_ns(1) turns the stencil kernel's pipeline
  waits into single non-blocking tests, so they give up on copies that are
  still in flight; the kernel stops its column after letting the issued
  copies land, the call returns FD_ERR_TIMEOUT, and the next call on the same
  context computes the same bits as before.
"""
import os

import numpy as np
import pytest

import workloads
from tests.gpu_util import require_cuda, to_dev

pytestmark = pytest.mark.gpu


def _problem(n=48, so=8, nt=60):
    shape = (n, n, n)
    h = (10.0, 10.0, 10.0)
    v = workloads.smooth_random(shape, 5, 4.0, 1.5, 3.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 6, h, 3.0)
    dt = workloads.cfl_dt(h, 3.0)
    c = (n / 2 - 0.5) * h[0]
    src = np.array([[[c, c, c]]], np.float32)
    xs = np.linspace(0.2, 0.8, 16) * (n - 1) * h[0]
    rec = np.stack([xs, np.full(16, c), np.full(16, 0.3 * (n - 1) * h[0])], -1)[None]
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None]
    return workloads.Workload("fail", shape, h, (0.0, 0.0, 0.0), so, dt, nt, m, damp,
                              src.astype(np.float32), wav.astype(np.float32),
                              rec.astype(np.float32))


def _run(torch, fd, w, u_init=None):
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp, u_init)
    rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
    torch.cuda.synchronize()
    return rec.cpu().numpy(), uf.cpu().numpy()


@pytest.mark.parametrize("kind", ["nan", "inf", "huge"])
def test_divergence_stops_the_time_loop_early(kind):
    """A NaN or Inf in u_init, or a finite state large enough to overflow in
    the first steps, gives FD_ERR_DIVERGED.  In statistics mode every stencil
    launch is timed: once the watchdog has fired the remaining launches
    return at once, so their total time is a small fraction of the clean
    run's."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError, _native
    w = _problem(n=256, so=8, nt=240)
    u0 = np.zeros((1, 2) + w.shape, np.float32)
    k = w.shape[0] // 2
    if kind == "nan":
        u0[0, 0, k, k, k] = np.nan
    elif kind == "inf":
        u0[0, 1, 3, 5, 7] = np.inf
    else:
        u0[0, 0, k - 2:k + 2, k - 2:k + 2, k - 2:k + 2] = 3e38
    _native.stats_enable(True)
    try:
        _native.stats_reset()
        _run(torch, fd, w)
        clean_ms, clean_n, _ = _native.stats_get("acoustic_step")
        _native.stats_reset()
        with pytest.raises(FdError) as e:
            _run(torch, fd, w, u_init=u0)
        bad_ms, bad_n, _ = _native.stats_get("acoustic_step")
    finally:
        _native.stats_enable(False)
    assert e.value.name == "FD_ERR_DIVERGED"
    assert clean_n == bad_n == w.nt - 1
    assert bad_ms < 0.5 * clean_ms, (bad_ms, clean_ms)
    # the context is still usable
    rec, uf = _run(torch, fd, w)
    assert np.all(np.isfinite(uf))


def test_tti_divergence_is_reported():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError
    w = workloads.tti_small(so=8, nt=40, n=32, nbl=4)
    p0 = np.zeros((1, 2) + w.shape, np.float32)
    p0[0, 0, 16, 16, 16] = np.nan
    g = fd.Grid(w.shape, w.spacing, w.origin)
    dev = to_dev(torch, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz, w.src_wav, w.rec_xyz,
                 w.damp, p0)
    m, e, d, th, ph, sx, sw, rx, dd, pi = dev
    with pytest.raises(FdError) as ex:
        fd.tti_forward(g, 8, w.dt, w.nt, m, e, d, th, ph, sx, sw, rx, damp=dd, p_init=pi)
    assert ex.value.name == "FD_ERR_DIVERGED"


def test_allocation_failure_is_reported_and_recovers():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError, _native
    from paper_1807_03032_gb300.serving import Engine
    w = _problem(n=40, so=4, nt=20)
    before = _native.load().fd_launch_count()
    os.environ["FDSWEEP_FAIL_ALLOC"] = "1"
    try:
        with pytest.raises(FdError) as e:
            _run(torch, fd, w)
        assert e.value.name == "FD_ERR_OOM"
        assert _native.load().fd_launch_count() == before  # nothing was launched
        g = fd.Grid(w.shape, w.spacing, w.origin)
        mt, dd = to_dev(torch, w.m, w.damp)
        with pytest.raises(FdError) as e:
            Engine(g, 4, w.dt, mt, dd, max_slots=2, max_nsrc=1, max_nrec=16)
        assert e.value.name == "FD_ERR_OOM"
    finally:
        del os.environ["FDSWEEP_FAIL_ALLOC"]
    rec, uf = _run(torch, fd, w)
    assert np.all(np.isfinite(uf)) and np.linalg.norm(rec) > 0


def test_bounded_wait_running_out_reports_timeout_and_the_context_survives():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError, _native
    lib = _native.load()
    w = _problem(n=64, so=16, nt=6)
    want = _run(torch, fd, w)
    lib.fd_set_wait_limit_ns(1)
    try:
        with pytest.raises(FdError) as e:
            _run(torch, fd, w)
    finally:
        lib.fd_set_wait_limit_ns(0)
    assert e.value.name == "FD_ERR_TIMEOUT"
    got = _run(torch, fd, w)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
