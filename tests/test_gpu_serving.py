"""Batch engine and continuous-batching server on the GPU: each shot's traces
are the same alone (acoustic_forward) and in the mix, and both match the FP64
oracle's traces for that shot."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, max_abs_rel, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def oracle_traces(shape, h, so, dt, m, damp, shot):
    """The oracle's traces of one shot run alone on the model."""
    nt, src, wav, rec = shot
    og = oracle.make_grid(shape, h)
    ref, _ = oracle.acoustic_forward(og, so, dt, nt, m, src[None], wav[None], rec[None],
                                     damp=damp)
    return ref[0]


def check_against_oracle(got, ref):
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(ref) > 0
    assert rel_l2(got, ref) <= TOL
    assert max_abs_rel(got, ref) <= TOL


def model_and_shots(n=40, seed=0, nshots=4, nts=(60, 44, 90, 30), so=8, h=10.0):
    shape = (n, n, n)
    rng = np.random.default_rng(seed)
    v = workloads.smooth_random(shape, seed + 3, 3.0, 1.5, 3.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 6, (h, h, h), 3.0)
    dt = workloads.cfl_dt((h, h, h), 3.0)
    ext = (n - 1) * h
    shots = []
    for i in range(nshots):
        nt = nts[i % len(nts)]
        src = rng.uniform(0.3, 0.7, (1, 3)) * ext
        xs = np.linspace(0.1 * ext, 0.9 * ext, 20)
        rec = np.stack([xs, np.full(20, 0.4 * ext + i * h), np.full(20, 0.2 * ext)], -1)
        wav = workloads.ricker(nt, dt, f0=0.03 + 0.005 * i)[:, None]
        shots.append((nt, src.astype(np.float32), wav.astype(np.float32), rec.astype(np.float32)))
    return shape, (h, h, h), so, dt, m, damp, shots


def standalone(torch, fd, g, so, dt, m, damp, shot):
    nt, src, wav, rec = shot
    s, w, r = to_dev(torch, src[None], wav[None], rec[None])
    out, _ = fd.acoustic_forward(g, so, dt, nt, m, s, w, r, damp=damp, return_final=False)
    torch.cuda.synchronize()
    return out[0].cpu().numpy()


def test_engine_shots_joining_mid_run_match_standalone():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300.serving import Engine
    shape, h, so, dt, m, damp, shots = model_and_shots()
    g = fd.Grid(shape, h)
    mt, dt_ = to_dev(torch, m, damp)
    eng = Engine(g, so, dt, mt, dt_, max_slots=3, max_nsrc=1, max_nrec=20)
    outs, slots = {}, {}
    # shot 0 and 1 at G = 0, shot 2 joins at G = 20, shot 3 reuses a freed slot later
    plan = {0: [0, 1], 20: [2]}
    G = 0
    done = []
    while len(done) < len(shots):
        for i in plan.get(G, []):
            nt, src, wav, rec = shots[i]
            s, w, r = to_dev(torch, src, wav, rec)
            outs[i] = torch.full((nt, 20), float("nan"), device="cuda")
            slots[i] = (eng.add_shot(nt, s, w, r, outs[i]), (s, w, r))
        eng.step(2)
        G += 2
        for i, (sl, _) in list(slots.items()):
            if eng.steps_left(sl) == 0:
                eng.release(sl)
                del slots[i]
                done.append(i)
                if i == 1 and 3 not in plan.get(G, []):
                    plan.setdefault(G, []).append(3)
    eng.sync()
    for i, shot in enumerate(shots):
        ref = standalone(torch, fd, g, so, dt, mt, dt_, shot)
        got = outs[i].cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) <= TOL, i
        check_against_oracle(got, oracle_traces(shape, h, so, dt, m, damp, shot))
    eng.close()


def test_server_mix_matches_standalone_and_baseline():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300.serving import Job, Model, Server, Shot, latency_stats, \
        one_shot_per_launch
    models, jobs, host_model = [], [], {}
    for mid, (n, seed) in enumerate(((40, 0), (32, 1))):
        shape, h, so, dt, m, damp, shots = model_and_shots(n=n, seed=seed, nshots=5)
        mt, dpt = to_dev(torch, m, damp)
        models.append((Model(mid, fd.Grid(shape, h), so, dt, mt, dpt), shots))
        host_model[mid] = (shape, h, so, dt, m, damp)
    rng = np.random.default_rng(2)
    t = 0.0
    job_shots = []
    for j in range(6):
        md, shots = models[j % 2]
        sel = [shots[k] for k in rng.choice(len(shots), size=rng.integers(1, 4), replace=False)]
        js = []
        for nt, src, wav, rec in sel:
            s, w, r = to_dev(torch, src, wav, rec)
            js.append(Shot(nt, s, w, r))
        jobs.append(Job(j, md, js, t))
        job_shots.append(sel)
        t += 0.002
    srv = Server(hbm_budget=8 << 30, max_slots=4, chunk=8, max_nsrc=1, max_nrec=20)
    done = srv.run(jobs)
    srv.close()
    assert len(done) == len(jobs)
    assert srv.max_concurrent_shots >= 2
    got = [[s.traces.cpu().numpy() for s in job.shots] for job in jobs]
    for job, gj, sel in zip(jobs, got, job_shots):
        md = job.model
        for shot, tr, host_shot in zip(job.shots, gj, sel):
            ref, _ = fd.acoustic_forward(md.grid, md.so, md.dt, shot.nt, md.m,
                                         shot.src_xyz[None], shot.src_wav[None],
                                         shot.rec_xyz[None], damp=md.damp, return_final=False)
            assert rel_l2(tr, ref[0].cpu().numpy()) <= TOL
            check_against_oracle(tr, oracle_traces(*host_model[md.model_id], host_shot))
    stats = latency_stats(jobs)
    assert stats["p99_s"] >= stats["p50_s"] > 0
    base = one_shot_per_launch(jobs)
    for job, gj in zip(base, got):
        for shot, tr in zip(job.shots, gj):
            assert rel_l2(shot.traces.cpu().numpy(), tr) <= TOL
