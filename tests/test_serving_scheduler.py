"""Scheduler logic of the continuous-batching server, on the CPU with a fake
engine (no GPU): every job finishes, admission keeps engines within the
memory budget, shots join running batches, results go to the right shot."""
import itertools

import pytest
import torch

from paper_1807_03032_gb300 import Grid
from paper_1807_03032_gb300.serving import Job, Model, Server, Shot, latency_stats


class FakeEvent:
    def query(self):
        return True


class FakeEngine:
    """Steps time on the host; a slot's 'trace' is filled with its shot tag."""

    created = 0
    live = 0

    def __init__(self, model, max_slots):
        FakeEngine.created += 1
        FakeEngine.live += 1
        self.model, self.max_slots = model, max_slots
        self.slots = {}
        self.G = 0
        self.max_active = 0

    def add_shot(self, nt, src_xyz, src_wav, rec_xyz, rec_out):
        free = [s for s in range(self.max_slots) if s not in self.slots]
        assert free, "no free slot"
        s = free[0]
        self.slots[s] = [self.G, nt, rec_out, float(src_wav[0, 0])]
        self.max_active = max(self.max_active, len(self.slots))
        return s

    def step(self, n):
        assert n % 2 == 0
        for s, (t0, nt, out, tag) in self.slots.items():
            lo, hi = self.G - t0, min(self.G - t0 + n, nt)
            if hi > lo:
                out[lo:hi] = tag
        self.G += n

    def steps_left(self, s):
        t0, nt, _, _ = self.slots[s]
        return max(0, t0 + nt - self.G)

    def release(self, s):
        del self.slots[s]

    def record_event(self):
        return FakeEvent()

    def close(self):
        FakeEngine.live -= 1


def make_jobs(n_jobs=12, seed=0):
    import random
    rnd = random.Random(seed)
    models = [Model(i, Grid((8, 8, 8), (1.0, 1.0, 1.0)), 4, 0.1, None, None) for i in range(3)]
    jobs, tag = [], itertools.count(1)
    t = 0.0
    for j in range(n_jobs):
        t += rnd.uniform(0.0, 0.004)
        md = models[rnd.randrange(3)]
        shots = []
        for _ in range(rnd.randint(1, 6)):
            nt = rnd.randrange(10, 200)
            wav = torch.full((nt, 1), float(next(tag)))
            shots.append(Shot(nt, torch.zeros(1, 3), wav, torch.zeros(5, 3)))
        jobs.append(Job(j, md, shots, t))
    return jobs


@pytest.mark.parametrize("budget_engines", [1, 2, 3])
def test_all_jobs_finish_within_budget(budget_engines):
    FakeEngine.created = FakeEngine.live = 0
    jobs = make_jobs()
    engines = []

    def factory(md):
        e = FakeEngine(md, 4)
        engines.append(e)
        return e

    srv = Server(hbm_budget=budget_engines * 100, max_slots=4, chunk=8, engine_factory=factory,
                 footprint_fn=lambda md: 100)
    done = srv.run(jobs)
    assert len(done) == len(jobs)
    assert srv.peak_used <= budget_engines * 100
    for job in jobs:
        assert job.done_at is not None and job.latency >= 0
        for shot in job.shots:
            tag = float(shot.src_wav[0, 0])
            assert torch.all(shot.traces == tag)
    assert max(e.max_active for e in engines) > 1  # shots share launches
    stats = latency_stats(jobs)
    assert stats["p99_s"] >= stats["p50_s"] >= 0
    srv.close()
    assert FakeEngine.live == 0


def test_model_larger_than_budget_is_rejected():
    jobs = make_jobs(2)
    srv = Server(hbm_budget=50, max_slots=4, chunk=8,
                 engine_factory=lambda md: FakeEngine(md, 4), footprint_fn=lambda md: 100)
    with pytest.raises(ValueError):
        srv.run(jobs)


def test_deliver_callback_receives_every_finished_shot_once():
    """With a deliver callback (the consumer of a long stream), every shot is
    handed over exactly once, after its traces are complete; the provided
    checksum_and_drop keeps the sum of squares and frees the traces."""
    from paper_1807_03032_gb300.serving import checksum_and_drop
    jobs = make_jobs(10, seed=3)
    seen = []

    def deliver(job, shot):
        tag = float(shot.src_wav[0, 0])
        assert torch.all(shot.traces == tag)
        want = float((shot.traces.double() ** 2).sum())
        seen.append(id(shot))
        checksum_and_drop(job, shot)
        assert shot.traces is None and float(shot.checksum) == want

    srv = Server(hbm_budget=300, max_slots=4, chunk=8,
                 engine_factory=lambda md: FakeEngine(md, 4), footprint_fn=lambda md: 100,
                 deliver=deliver)
    srv.run(jobs)
    srv.close()
    all_shots = [id(s) for j in jobs for s in j.shots]
    assert sorted(seen) == sorted(all_shots)
