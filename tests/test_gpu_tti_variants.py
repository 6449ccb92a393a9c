"""GPU parity of the TTI ablation variants (tti_forward_opts) against the FP64
oracle: staggered first derivatives, (p + r)/2 receivers, and the recompute
scheme (no first-derivative temporaries)."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def run_pair(w, deriv="centred", receiver="p", scheme="two_pass", p_init=None, r_init=None):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    g = fd.Grid(w.shape, w.spacing, w.origin)
    dev = to_dev(torch, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz, w.src_wav, w.rec_xyz,
                 w.damp, p_init, r_init)
    m, e, d, th, ph, sx, sw, rx, dd, pi, ri = dev
    rec, pf, rf = fd.tti_forward(g, w.so, w.dt, w.nt, m, e, d, th, ph, sx, sw, rx, damp=dd,
                                 p_init=pi, r_init=ri, deriv=deriv, receiver=receiver,
                                 scheme=scheme)
    torch.cuda.synchronize()
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    ref = oracle.tti_forward(og, w.so, w.dt, w.nt, w.m, w.eps, w.delta, w.theta, w.phi,
                             w.src_xyz, w.src_wav, w.rec_xyz, damp=w.damp, p_init=p_init,
                             r_init=r_init, deriv=deriv, receiver=receiver)
    return (rec.cpu().numpy(), pf.cpu().numpy(), rf.cpu().numpy()), ref


def check(got, ref):
    (rec, pf, rf), (rref, pref, qref) = got, ref
    assert np.linalg.norm(rref) > 0
    assert rel_l2(pf, pref) <= TOL
    assert rel_l2(rf, qref) <= TOL
    assert rel_l2(rec, rref) <= TOL


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_staggered_two_pass_parity(so):
    w = workloads.tti_small(so=so, nt=80)
    check(*run_pair(w, deriv="staggered"))


@pytest.mark.parametrize("deriv", ["centred", "staggered"])
def test_mean_receivers_parity(deriv):
    w = workloads.tti_small(so=8, nt=80)
    got, ref = run_pair(w, deriv=deriv, receiver="mean")
    check(got, ref)
    # the reading matters: p-only traces differ from the mean traces
    got_p, _ = run_pair(w, deriv=deriv)
    assert rel_l2(got[0], got_p[0]) > 1e-3


@pytest.mark.parametrize("so,deriv", [(4, "centred"), (8, "staggered"), (12, "centred"),
                                      (16, "staggered")])
def test_recompute_scheme_parity(so, deriv):
    w = workloads.tti_small(so=so, nt=60)
    check(*run_pair(w, deriv=deriv, scheme="recompute"))


@pytest.mark.parametrize("so", [2, 4])
def test_two_pass_centred_small_orders(so):
    """The two-pass scheme where the automatic choice is the fused one."""
    w = workloads.tti_small(so=so, nt=60)
    check(*run_pair(w, scheme="two_pass"))


@pytest.mark.parametrize("so,deriv", [(2, "centred"), (4, "centred"), (4, "staggered"),
                                      (8, "centred"), (8, "staggered")])
def test_fused_scheme_parity(so, deriv):
    """One kernel per step with the temporaries in shared memory."""
    w = workloads.tti_small(so=so, nt=60)
    check(*run_pair(w, deriv=deriv, scheme="fused"))


@pytest.mark.parametrize("so", [4, 8])
def test_fused_scheme_interior_and_chunks(so):
    """80^3 (interior tiles away from every boundary, z split into chunks)."""
    w = workloads.tti_small(so=so, nt=40, n=80)
    check(*run_pair(w, scheme="fused"))


def test_fused_scheme_rejects_wide_stencils():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    w = workloads.tti_small(so=12, nt=4)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, e, d, th, ph, sx, sw, rx = to_dev(torch, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz,
                                         w.src_wav, w.rec_xyz)
    with pytest.raises(_native.FdError):
        fd.tti_forward(g, 12, w.dt, w.nt, m, e, d, th, ph, sx, sw, rx, scheme="fused")


@pytest.mark.parametrize("scheme", ["two_pass", "recompute", "fused"])
def test_ragged_multishot_staggered_mean(scheme):
    """Ragged box, anisotropic spacing, two shots, random initial fields,
    theta over [0, pi] (n_z of either sign), staggered derivatives and mean
    receivers together."""
    shape = (27, 21, 35)
    h = (10.0, 12.0, 9.0)
    o = (5.0, -40.0, 100.0)
    rng = np.random.default_rng(15)
    eps = rng.uniform(0.0, 0.3, shape)
    delta = np.minimum(rng.uniform(-0.1, 0.2, shape), eps)
    theta = rng.uniform(0.0, np.pi, shape)
    phi = rng.uniform(-np.pi, np.pi, shape)
    v = workloads.two_layer_velocity(shape, 1.8, 3.0)
    dt = 0.9 * workloads.cfl_dt(h, 3.0, eps_max=0.3)
    nt, nshots = 30, 2
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    src = o + rng.uniform(0.1, 0.9, (nshots, 2, 3)) * ext
    rec = o + rng.uniform(0.0, 1.0, (nshots, 11, 3)) * ext
    wav = rng.standard_normal((nshots, nt, 2))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    w = workloads.Workload("tti-ragged", shape, h, o, 8, dt, nt, workloads.slowness_squared(v),
                           workloads.damping_profile(shape, 4, h, 3.0), f32(src), f32(wav),
                           f32(rec), eps=f32(eps), delta=f32(delta), theta=f32(theta),
                           phi=f32(phi))
    p_init = 1e-2 * workloads.random_wavefields(shape, 21, nshots=nshots, sigma=2.0)
    r_init = 1e-2 * workloads.random_wavefields(shape, 22, nshots=nshots, sigma=2.0)
    check(*run_pair(w, deriv="staggered", receiver="mean", scheme=scheme, p_init=p_init,
                    r_init=r_init))


def test_options_out_of_range_rejected():
    torch = require_cuda()
    import ctypes
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    w = workloads.tti_small(so=4, nt=4)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, e, d, th, ph, sx, sw, rx = to_dev(torch, w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz,
                                         w.src_wav, w.rec_xyz)
    rec = torch.empty((1, w.nt, w.rec_xyz.shape[1]), device="cuda")
    lib = _native.load()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    for bad in ((2, 0, 0), (0, 5, 0), (0, 0, 7), (0, 0, -2)):
        opts = _native.FdTtiOptions(*bad)
        st = lib.tti_forward_opts(g.struct(), 4, w.dt, w.nt, 1, P(m), None, P(e), P(d), P(th),
                                  P(ph), 1, P(sx), P(sw), w.rec_xyz.shape[1], P(rx), P(rec),
                                  None, None, None, None, ctypes.byref(opts), None)
        assert st == -1, bad


@pytest.mark.parametrize("so,deriv", [(4, "staggered"), (16, "centred")])
def test_recompute_interior_blocks_parity(so, deriv):
    """80^3: the recompute kernel's unchecked interior blocks (all taps inside
    the grid) as well as its boundary blocks are exercised."""
    w = workloads.tti_small(so=so, nt=40, n=80)
    check(*run_pair(w, deriv=deriv, scheme="recompute"))
