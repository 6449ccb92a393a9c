"""GPU parity of the acoustic forward run with the damping given as a 3-D
field (acoustic_forward_opts with FD_DAMP_FIELD) against the oracle's 3-D
damping path, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, max_abs_rel, rel_l2, require_cuda, to_dev
from tests.test_oracle_damp_field import _sponge

pytestmark = pytest.mark.gpu


def _run(torch, fd, w, damp, u_init=None, layout="field"):
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, damp, u_init)
    rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui,
                                  damp_layout=layout)
    torch.cuda.synchronize()
    return rec.cpu().numpy(), uf.cpu().numpy()


def _oracle(w, damp, u_init=None, layout="field"):
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    return oracle.acoustic_forward(og, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav, w.rec_xyz,
                                   damp=damp, u_init=u_init, damp_layout=layout)


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_ragged_multishot_non_separable_sponge(so):
    from tests.test_gpu_acoustic import ragged_problem
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w, u_init = ragged_problem(so)
    damp = _sponge(w.shape, w.spacing, 6, 0.5, 11)
    rec, uf = _run(torch, fd, w, damp, u_init)
    rref, uref = _oracle(w, damp, u_init)
    assert rel_l2(uf, uref) <= TOL and rel_l2(rec, rref) <= TOL
    assert max_abs_rel(uf, uref) <= TOL


@pytest.mark.parametrize("so", [4, 16])
def test_small_workload_with_a_non_separable_sponge(so):
    """The 64^3 two-layer workload for 400 steps with its 10-point border
    replaced by a non-separable absorbing mask of the same strength."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_small(so=so, nt=400)
    d0 = float(np.max(w.damp))
    damp = _sponge(w.shape, w.spacing, w.nbl, d0, 12)
    rec, uf = _run(torch, fd, w, damp)
    rref, uref = _oracle(w, damp)
    assert np.linalg.norm(rref) > 0
    for got, ref in ((rec, rref), (uf, uref)):
        assert rel_l2(got, ref) <= TOL
        assert max_abs_rel(got, ref) <= TOL


def test_separable_field_agrees_with_the_profiles():
    """A 3-D field equal to the sum of the per-axis profiles gives the
    profile path's result to FP32 rounding (the two paths form the damping
    factor with different roundings), and both match the oracle."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_small(so=8, nt=150)
    n = w.shape[0]
    dx, dy, dz = w.damp[:n], w.damp[n:2 * n], w.damp[2 * n:]
    field = (dz[:, None, None].astype(np.float64) + dy[None, :, None] + dx[None, None, :])
    field = np.ascontiguousarray(field, dtype=np.float32)
    rf, uf = _run(torch, fd, w, field)
    ra, ua = _run(torch, fd, w, w.damp, layout="axes")
    assert rel_l2(uf, ua) <= 1e-6
    rref, uref = _oracle(w, w.damp, layout="axes")
    assert rel_l2(uf, uref) <= TOL and rel_l2(ua, uref) <= TOL


def test_damp_field_errors():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError
    w = workloads.acoustic_small(so=4, nt=10)
    damp = _sponge(w.shape, w.spacing, 10, 0.1, 13)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, damp)
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, w.dt, w.nt, m, sx, sw, rx, damp=dd, damp_layout="field",
                            storage="f16")
    assert e.value.name == "FD_ERR_ARG"
    bad = dd.clone()
    bad[5, 6, 7] = -1.0
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, w.dt, w.nt, m, sx, sw, rx, damp=bad, damp_layout="field")
    assert e.value.name == "FD_ERR_ARG"
    rec, _ = fd.acoustic_forward(g, 4, w.dt, w.nt, m, sx, sw, rx, damp=dd, damp_layout="field")
    assert torch.isfinite(rec).all()
