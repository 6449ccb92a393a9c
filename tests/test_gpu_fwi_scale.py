"""The FWI gradient at a reduced version of the benchmark's gradient workload
(layered true model, smoothed initial model, shots on a surface grid, a full
surface receiver plane, so 8, checkpointing), against the FP64 oracle's
gradient, and a Taylor test of the GPU gradient on the GPU's own forward map.

The gradient workload of the benchmark is 256^3, 16 shots, nt 2000, a
checkpoint every 45 steps; here the grid is 96^3 with a 16-point border, 4
shots, nt 400 and a checkpoint every 20 steps, and the shots are forced into
batches of 2 so that the batched gradient accumulates over several batches.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, max_abs_rel, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def _reduced_workload():
    true, init = workloads.fwi_layered(n=96, so=8, nt=400, nshots=4, nbl=16,
                                       receivers_per_side=48, smooth_sigma=4.0)
    return true, init


def _forward(torch, fd, w, m):
    g = fd.Grid(w.shape, w.spacing, w.origin)
    mt, sx, sw, rx, dd = to_dev(torch, m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp)
    d, _ = fd.acoustic_forward(g, w.so, w.dt, w.nt, mt, sx, sw, rx, damp=dd, return_final=False)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_gradient_matches_oracle_over_several_shot_batches():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    true, init = _reduced_workload()
    dobs = _forward(torch, fd, true, true.m)
    dpred = _forward(torch, fd, init, init.m)
    resid = (dpred - dobs).astype(np.float32)
    g = fd.Grid(init.shape, init.spacing, init.origin)
    mt, sx, sw, rx, dd, rr = to_dev(torch, init.m, init.src_xyz, init.src_wav, init.rec_xyz,
                                    init.damp, resid)
    os.environ["FDSWEEP_GRAD_BATCH"] = "2"
    try:
        grad = fd.acoustic_gradient(g, 8, init.dt, init.nt, mt, sx, sw, rx, rr, damp=dd,
                                    checkpoint_every=20)
        torch.cuda.synchronize()
    finally:
        del os.environ["FDSWEEP_GRAD_BATCH"]
    grad = grad.cpu().numpy()
    og = oracle.make_grid(init.shape, init.spacing, init.origin)
    ref = oracle.acoustic_gradient(og, 8, init.dt, init.nt, init.m, init.src_xyz, init.src_wav,
                                   init.rec_xyz, resid, damp=init.damp)
    assert np.linalg.norm(ref) > 0
    assert rel_l2(grad, ref) <= TOL
    assert max_abs_rel(grad, ref) <= TOL


def test_taylor_expansion_of_the_gpu_objective():
    """J(m) = 1/2 ||d(m) - d_obs||^2 with the GPU forward model (traces in
    FP32, J summed in FP64): along the model update dm = m_true - m0 the
    first-order remainder |J(m + h dm) - J(m)| halves with h and the
    second-order one |J(m + h dm) - J(m) - h <g, dm>| quarters, with g the GPU
    gradient."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    true, init = _reduced_workload()
    dobs = _forward(torch, fd, true, true.m).astype(np.float64)

    def J(m):
        r = _forward(torch, fd, init, m).astype(np.float64) - dobs
        return 0.5 * float(np.sum(r * r))

    m0 = init.m.astype(np.float64)
    J0 = J(init.m)
    resid = (_forward(torch, fd, init, init.m) - dobs).astype(np.float32)
    g = fd.Grid(init.shape, init.spacing, init.origin)
    mt, sx, sw, rx, dd, rr = to_dev(torch, init.m, init.src_xyz, init.src_wav, init.rec_xyz,
                                    init.damp, resid)
    grad = fd.acoustic_gradient(g, 8, init.dt, init.nt, mt, sx, sw, rx, rr, damp=dd,
                                checkpoint_every=20)
    torch.cuda.synchronize()
    grad = grad.cpu().numpy().astype(np.float64)
    dm = true.m.astype(np.float64) - m0
    gdm = float(np.sum(grad * dm))
    assert gdm < 0  # the update toward the true model descends
    hs = (0.1, 0.05, 0.025)
    r1, r2 = [], []
    for h in hs:
        Jh = J(np.ascontiguousarray(m0 + h * dm, dtype=np.float32))
        r1.append(abs(Jh - J0))
        r2.append(abs(Jh - J0 - h * gdm))
    s1 = [np.log2(r1[i] / r1[i + 1]) for i in range(2)]
    s2 = [np.log2(r2[i] / r2[i + 1]) for i in range(2)]
    assert all(0.8 <= s <= 1.2 for s in s1), (r1, s1)
    assert all(1.6 <= s <= 2.4 for s in s2), (r2, s2)
    assert r2[-1] < 0.05 * r1[-1]
