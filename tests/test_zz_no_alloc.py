"""acoustic_forward_noalloc: the allocation-free acoustic forward model.

For callers that cannot allocate device memory (a fixed memory budget, a
foreign allocator that owns the device memory, a service that must not hit
out-of-memory mid-request), the library offers a variant of acoustic_forward
whose workspace lives in a fixed device array instead of a per-call
allocation.  These tests call it through the C ABI and check it against
acoustic_forward on the same inputs, twice in a row (the array keeps the
previous call's contents, so the second call shows that every call starts
from a clean state).  The call runs acoustic_forward's schedule with the same
kernels, launch configuration and in-kernel injection order, so with at most
16 sources per shot its results are bit-identical to acoustic_forward's.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import workloads
from tests.gpu_util import TOL, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def _call_noalloc(torch, lib, g, w, dev, u_init=None):
    m, sx, sw, rx, dd = dev
    nshots, nsrc, nrec = w.src_xyz.shape[0], w.src_xyz.shape[1], w.rec_xyz.shape[1]
    # outputs pre-filled with NaN: every element must be written by the call
    rec = torch.full((nshots, w.nt, nrec), float("nan"), device="cuda")
    uf = torch.full((nshots, 2) + tuple(w.shape), float("nan"), device="cuda")
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    st = lib.acoustic_forward_noalloc(
        g.struct(), w.so, w.dt, w.nt, nshots, ptr(m), ptr(dd), nsrc, ptr(sx), ptr(sw), nrec,
        ptr(rx), ptr(rec), ptr(u_init), ptr(uf),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    from paper_1807_03032_gb300 import _native
    _native.check(st)
    torch.cuda.synchronize()
    return rec.cpu().numpy(), uf.cpu().numpy()


@pytest.mark.parametrize("so", [4, 16])
def test_noalloc_matches_acoustic_forward_on_two_calls_in_a_row(so):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    lib = _native.load()
    w = workloads.acoustic_small(so=so, nt=60)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    dev = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp)
    m, sx, sw, rx, dd = dev
    rec_ref, uf_ref = fd.acoustic_forward(g, so, w.dt, w.nt, m, sx, sw, rx, damp=dd)
    rec_ref, uf_ref = rec_ref.cpu().numpy(), uf_ref.cpu().numpy()
    for _ in range(2):
        rec, uf = _call_noalloc(torch, lib, g, w, dev)
        assert np.all(np.isfinite(uf)) and np.all(np.isfinite(rec))
        assert rel_l2(uf, uf_ref) <= TOL
        assert rel_l2(rec, rec_ref, floor=1e-3 * np.linalg.norm(rec_ref)) <= TOL
        np.testing.assert_array_equal(uf, uf_ref)
        np.testing.assert_array_equal(rec, rec_ref)


def test_noalloc_multishot_with_initial_state_twice():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    lib = _native.load()
    shape = (30, 22, 37)
    h = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(4)
    v = workloads.smooth_random(shape, 4, 3.0, 1.5, 3.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 4, h, 3.0)
    dt = 0.9 * workloads.cfl_dt(h, 3.0)
    nt, nshots = 40, 2
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    src = (rng.uniform(0.1, 0.9, (nshots, 2, 3)) * ext).astype(np.float32)
    rec = (rng.uniform(0.0, 1.0, (nshots, 9, 3)) * ext).astype(np.float32)
    wav = rng.standard_normal((nshots, nt, 2)).astype(np.float32)
    w = workloads.Workload("multi", shape, h, (0.0, 0.0, 0.0), 8, dt, nt, m, damp, src, wav, rec)
    u_init = 1e-2 * workloads.random_wavefields(shape, 9, nshots=nshots, sigma=2.0)
    g = fd.Grid(shape, h)
    dev = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp)
    ui, = to_dev(torch, u_init)
    m_, sx, sw, rx, dd = dev
    rec_ref, uf_ref = fd.acoustic_forward(g, 8, dt, nt, m_, sx, sw, rx, damp=dd, u_init=ui)
    rec_ref, uf_ref = rec_ref.cpu().numpy(), uf_ref.cpu().numpy()
    for _ in range(2):
        r, uf = _call_noalloc(torch, lib, g, w, dev, u_init=ui)
        assert rel_l2(uf, uf_ref) <= TOL
        assert rel_l2(r, rec_ref) <= TOL
        np.testing.assert_array_equal(uf, uf_ref)
        np.testing.assert_array_equal(r, rec_ref)


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError, _native
    lib = _native.load()
    w = workloads.acoustic_small(so=4, nt=4)
    big = (256, 256, 256)  # 3 x 64 MiB of workspace > the fixed scratch
    g = fd.Grid(big, w.spacing, w.origin)
    m = torch.full(big, float(w.m.max()), device="cuda")
    st = lib.acoustic_forward_noalloc(g.struct(), 4, w.dt, 4, 1, ctypes.c_void_p(m.data_ptr()),
                                      None, 0, None, None, 0, None, None, None, None, None)
    with pytest.raises(FdError) as e:
        _native.check(st)
    assert e.value.name == "FD_ERR_ARG" and "scratch" in str(e.value)
