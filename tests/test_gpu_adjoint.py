"""GPU adjoint, FWI gradient and autograd against the FP64 oracle (through the
C ABI), plus the dot-product test in FP32."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def problem(so=4, nt=40, nshots=2, seed=0, shape=(22, 18, 27), nbl=4):
    h = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(seed)
    v = workloads.smooth_random(shape, seed + 1, 2.5, 1.5, 2.5)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, nbl, h, 2.5)
    dt = workloads.cfl_dt(h, 2.5)
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    src = (rng.uniform(0.25, 0.75, (nshots, 2, 3)) * ext).astype(np.float32)
    rec = (rng.uniform(0.05, 0.95, (nshots, 9, 3)) * ext).astype(np.float32)
    wav = np.stack([workloads.ricker(nt, dt, f0=0.03), workloads.ricker(nt, dt, f0=0.02)], -1)
    wav = np.repeat(wav[None], nshots, 0).astype(np.float32)
    return shape, h, so, dt, nt, m, damp, src, wav, rec


@pytest.mark.parametrize("so,nt", [(4, 20), (8, 45), (16, 40)])
def test_adjoint_matches_oracle(so, nt):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    shape, h, so, dt, nt, m, damp, src, wav, rec = problem(so=so, nt=nt)
    dd = np.random.default_rng(7).standard_normal((src.shape[0], nt, rec.shape[1])).astype(np.float32)
    g = fd.Grid(shape, h)
    mt, dampt, srct, rect, ddt = to_dev(torch, m, damp, src, rec, dd)
    qa = fd.acoustic_adjoint(g, so, dt, nt, mt, srct, rect, ddt, damp=dampt)
    torch.cuda.synchronize()
    qa = qa.cpu().numpy()
    ref = oracle.acoustic_adjoint(oracle.make_grid(shape, h), so, dt, nt, m, src, rec, dd,
                                  damp=damp)
    assert rel_l2(qa, ref) <= TOL
    assert np.all(qa[:, -1] == 0)


def test_dot_product_fp32():
    """<F q, d> = <F^T d, q> to 1e-5 with the GPU forward and adjoint (64^3,
    so = 8, 100 steps, damping border)."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_small(so=8, nt=100)
    rng = np.random.default_rng(11)
    q = rng.standard_normal(w.src_wav.shape).astype(np.float32)
    rec = np.concatenate([w.rec_xyz, w.src_xyz + np.float32(17.0)], axis=1)
    dd = rng.standard_normal((1, w.nt, rec.shape[1])).astype(np.float32)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    mt, dampt, srct, rect, qt, ddt = to_dev(torch, w.m, w.damp, w.src_xyz, rec, q, dd)
    d, _ = fd.acoustic_forward(g, 8, w.dt, w.nt, mt, srct, qt, rect, damp=dampt,
                               return_final=False)
    qa = fd.acoustic_adjoint(g, 8, w.dt, w.nt, mt, srct, rect, ddt, damp=dampt)
    torch.cuda.synchronize()
    lhs = float(np.vdot(d.cpu().numpy().astype(np.float64), dd.astype(np.float64)))
    rhs = float(np.vdot(q.astype(np.float64), qa.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("so", [4, 12])
def test_gradient_matches_oracle(so):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    shape, h, so, dt, nt, m, damp, src, wav, rec = problem(so=so, nt=36)
    dd = np.random.default_rng(3).standard_normal((src.shape[0], nt, rec.shape[1])).astype(np.float32)
    g = fd.Grid(shape, h)
    mt, dampt, srct, wavt, rect, ddt = to_dev(torch, m, damp, src, wav, rec, dd)
    gr = fd.acoustic_gradient(g, so, dt, nt, mt, srct, wavt, rect, ddt, damp=dampt,
                              checkpoint_every=5)
    torch.cuda.synchronize()
    ref = oracle.acoustic_gradient(oracle.make_grid(shape, h), so, dt, nt, m, src, wav, rec, dd,
                                   damp=damp)
    assert rel_l2(gr.cpu().numpy(), ref) <= TOL


def test_gradient_independent_of_checkpoint_interval():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    shape, h, so, dt, nt, m, damp, src, wav, rec = problem(so=8, nt=30, nshots=1)
    dd = np.random.default_rng(4).standard_normal((1, nt, rec.shape[1])).astype(np.float32)
    g = fd.Grid(shape, h)
    mt, dampt, srct, wavt, rect, ddt = to_dev(torch, m, damp, src, wav, rec, dd)
    outs = []
    for k in (1, 4, 0, 29, 100):
        gr = fd.acoustic_gradient(g, so, dt, nt, mt, srct, wavt, rect, ddt, damp=dampt,
                                  checkpoint_every=k)
        torch.cuda.synchronize()
        outs.append(gr.cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_autograd_gradients_and_central_difference():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300.autograd import acoustic_modeling
    shape, h, so, dt, nt, m_true, damp, src, wav, rec = problem(so=8, nt=50, nshots=2)
    g = fd.Grid(shape, h)
    m0 = workloads.slowness_squared(1.0 / np.sqrt(m_true.astype(np.float64)) * 1.04)
    mt_true, m0t, dampt, srct, wavt, rect = to_dev(torch, m_true, m0, damp, src, wav, rec)
    with torch.no_grad():
        dobs = acoustic_modeling(mt_true, wavt, g, so, dt, srct, rect, dampt)
    m = m0t.clone().requires_grad_(True)
    q = wavt.clone().requires_grad_(True)
    d = acoustic_modeling(m, q, g, so, dt, srct, rect, dampt, checkpoint_every=7)
    J = 0.5 * ((d - dobs) ** 2).sum()
    gm, gq = torch.autograd.grad(J, (m, q))
    resid = (d - dobs).detach().contiguous()
    gm_ref = oracle.acoustic_gradient(oracle.make_grid(shape, h), so, dt, nt, m0, src, wav, rec,
                                      resid.cpu().numpy(), damp=damp)
    assert rel_l2(gm.cpu().numpy(), gm_ref) <= TOL
    gq_ref = oracle.acoustic_adjoint(oracle.make_grid(shape, h), so, dt, nt, m0, src, rec,
                                     resid.cpu().numpy(), damp=damp)
    assert rel_l2(gq.cpu().numpy(), gq_ref) <= TOL
    # central difference of J along a smooth perturbation, in FP32 on the GPU
    dm = torch.from_numpy(workloads.smooth_random(shape, 5, 2.0, -1.0, 1.0).astype(np.float32)).cuda()
    dm *= float(m0t.mean()) * 2e-3

    def J_of(mm):
        with torch.no_grad():
            dd_ = acoustic_modeling(mm.contiguous(), wavt, g, so, dt, srct, rect, dampt)
            return 0.5 * float(((dd_ - dobs).double() ** 2).sum())

    fd_est = (J_of(m0t + dm) - J_of(m0t - dm)) / 2.0
    an = float((gm.double() * dm.double()).sum())
    assert abs(fd_est - an) <= 2e-2 * abs(an), (fd_est, an)


def test_gradient_shot_batches_sum_the_shots(monkeypatch):
    """Five shots processed in batches of 2, 2, 1 and in one batch give the
    same gradient (up to the order of FP32 accumulation), and it matches the
    oracle."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    shape, h, so, dt, nt, m, damp, src, wav, rec = problem(so=8, nt=24, nshots=5, seed=5)
    dd = np.random.default_rng(9).standard_normal((5, nt, rec.shape[1])).astype(np.float32)
    g = fd.Grid(shape, h)
    mt, dampt, srct, wavt, rect, ddt = to_dev(torch, m, damp, src, wav, rec, dd)
    whole = fd.acoustic_gradient(g, so, dt, nt, mt, srct, wavt, rect, ddt, damp=dampt,
                                 checkpoint_every=7).cpu().numpy()
    monkeypatch.setenv("FDSWEEP_GRAD_BATCH", "2")
    parts = fd.acoustic_gradient(g, so, dt, nt, mt, srct, wavt, rect, ddt, damp=dampt,
                                 checkpoint_every=7).cpu().numpy()
    torch.cuda.synchronize()
    assert rel_l2(parts, whole) <= 1e-6
    ref = oracle.acoustic_gradient(oracle.make_grid(shape, h), so, dt, nt, m, src, wav, rec, dd,
                                   damp=damp)
    assert rel_l2(whole, ref) <= TOL
