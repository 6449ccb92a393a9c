"""Serving loop with continuous batching over the batch engine.

Requests ("jobs") are seismic experiments: one velocity model (grid, so, dt,
m, damp) and 1..32 shots, each with its own source, wavelet, receivers and
number of time steps.  The server keeps one batch engine per model
(``fd_engine_*`` in the C ABI): the model's shots are slots of that engine and
advance together, one stencil launch per time step over all active slots (the
shot is the outer dimension), in graph-captured chunks.  Between chunks,
finished shots are delivered and their slots freed, and queued shots join
immediately -- also while other shots of the same engine are mid-run -- so
the batch is continuous rather than formed once.  Engines run on their own
streams, so different models overlap on the device.  A new engine is admitted
only if its device footprint fits the memory budget; otherwise its jobs wait
until an idle engine is retired.  Wavefields never leave the device; only the
traces are delivered.

``one_shot_per_launch`` is the comparison path: every shot of every job runs
as its own ``acoustic_forward`` call, in arrival order.

Everything numeric runs in the library's kernels; this module schedules.
"""
from __future__ import annotations

import ctypes
import math
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import _native, acoustic_forward
from . import Grid


# ---------------------------------------------------------------- engine

class Engine:
    """Python handle of one ``fd_engine`` (all tensors are CUDA tensors)."""

    def __init__(self, grid: Grid, so, dt, m, damp, max_slots, max_nsrc, max_nrec):
        import torch
        self.torch = torch
        self.grid, self.so, self.dt = grid, so, dt
        self.max_slots, self.max_nsrc, self.max_nrec = max_slots, max_nsrc, max_nrec
        self._keep = [m, damp]
        h = ctypes.c_void_p()
        lib = _native.load()
        _native.check(lib.fd_engine_create(grid.struct(), int(so), float(dt),
                                           m.data_ptr(), None if damp is None else damp.data_ptr(),
                                           max_slots, max_nsrc, max_nrec, ctypes.byref(h)))
        self.h = h
        sp = ctypes.c_void_p()
        _native.check(lib.fd_engine_stream(h, ctypes.byref(sp)))
        self.stream = torch.cuda.ExternalStream(sp.value)
        self.slot_refs = {}

    @staticmethod
    def footprint(grid: Grid, max_slots, max_nsrc, max_nrec) -> int:
        b = ctypes.c_int64()
        _native.check(_native.load().fd_engine_footprint(grid.struct(), max_slots, max_nsrc,
                                                         max_nrec, ctypes.byref(b)))
        return int(b.value)

    def add_shot(self, nt, src_xyz, src_wav, rec_xyz, rec_out) -> int:
        slot = ctypes.c_int()
        _native.check(_native.load().fd_engine_add_shot(
            self.h, int(nt), int(src_xyz.shape[0]), src_xyz.data_ptr(), src_wav.data_ptr(),
            int(rec_xyz.shape[0]), rec_xyz.data_ptr(), rec_out.data_ptr(), ctypes.byref(slot)))
        self.slot_refs[slot.value] = (src_xyz, src_wav, rec_xyz, rec_out)
        return slot.value

    def step(self, nsteps):
        _native.check(_native.load().fd_engine_step(self.h, int(nsteps)))

    def steps_left(self, slot) -> int:
        a = ctypes.c_int()
        left = ctypes.c_int64()
        _native.check(_native.load().fd_engine_shot_status(self.h, slot, ctypes.byref(a),
                                                           ctypes.byref(left)))
        return int(left.value) if a.value else -1

    def release(self, slot):
        _native.check(_native.load().fd_engine_release(self.h, slot))
        self.slot_refs.pop(slot, None)

    def record_event(self):
        """An event recorded on the engine's stream (query() -> reached)."""
        ev = self.torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def sync(self):
        _native.check(_native.load().fd_engine_sync(self.h))

    def close(self):
        if self.h:
            _native.check(_native.load().fd_engine_destroy(self.h))
            self.h = None


# ---------------------------------------------------------------- requests

@dataclass(eq=False)
class Model:
    """A velocity model and its discretisation (shared by a job's shots)."""

    model_id: int
    grid: Grid
    so: int
    dt: float
    m: object          # CUDA tensor [nz][ny][nx]
    damp: object       # CUDA tensor [nx+ny+nz] or None


@dataclass(eq=False)
class Shot:
    nt: int
    src_xyz: object    # CUDA tensor [nsrc][3]
    src_wav: object    # CUDA tensor [nt][nsrc]
    rec_xyz: object    # CUDA tensor [nrec][3]
    traces: object = None
    done_at: Optional[float] = None
    checksum: object = None  # set by a deliver callback that drops the traces


def checksum_and_drop(job, shot):
    """A deliver callback for long streams: keeps the sum of squares of the
    shot's traces (a device scalar) and frees the traces, so that the device
    memory held by delivered results stays bounded."""
    shot.checksum = shot.traces.double().square().sum()
    shot.traces = None


@dataclass(eq=False)
class Job:
    job_id: int
    model: Model
    shots: list
    arrival: float     # seconds after the start of the run
    done_at: Optional[float] = None

    @property
    def latency(self):
        return None if self.done_at is None else self.done_at - self.arrival


@dataclass
class _EngineState:
    engine: object
    model: Model
    footprint: int
    queue: deque = field(default_factory=deque)      # (job, shot)
    running: dict = field(default_factory=dict)      # slot -> (job, shot)
    finishing: set = field(default_factory=set)      # slots whose last step is enqueued
    pending: list = field(default_factory=list)      # (event, [(slot, job, shot)])
    idle_since: Optional[float] = None


class Server:
    """Continuous-batching server over per-model batch engines.

    hbm_budget: bytes of device memory engines may use together (admission).
    max_slots: slots per engine (shots of one model in flight).
    chunk: time steps per engine step between scheduling decisions (even).
    engine_factory: builds an engine for a model (tests inject a fake).
    deliver: called as deliver(job, shot) once a shot's traces are complete
    (the consumer; by default the traces stay on the shot).
    """

    def __init__(self, hbm_budget, max_slots=32, chunk=32, max_nsrc=1, max_nrec=16384,
                 engine_factory: Optional[Callable] = None, footprint_fn: Optional[Callable] = None,
                 clock: Callable = time.perf_counter, deliver: Optional[Callable] = None):
        self.deliver = deliver
        self.budget = int(hbm_budget)
        self.max_slots = max_slots
        self.chunk = chunk + (chunk & 1)
        self.max_nsrc, self.max_nrec = max_nsrc, max_nrec
        self.engine_factory = engine_factory or (
            lambda md: Engine(md.grid, md.so, md.dt, md.m, md.damp, self.max_slots,
                              self.max_nsrc, self.max_nrec))
        self.footprint_fn = footprint_fn or (
            lambda md: Engine.footprint(md.grid, self.max_slots, self.max_nsrc, self.max_nrec))
        self.clock = clock
        self.engines = {}          # model_id -> _EngineState
        self.waiting = deque()     # jobs whose engine is not admitted yet
        self.used = 0
        self.jobs_done = []
        self.t0 = None
        self.peak_used = 0
        self.max_concurrent_shots = 0

    # ------------------------------------------------------------ scheduling
    def _admit(self, job, now):
        st = self.engines.get(job.model.model_id)
        if st is None:
            need = self.footprint_fn(job.model)
            if need > self.budget:
                raise ValueError(f"model {job.model.model_id} needs {need} bytes, more than "
                                 f"the whole budget {self.budget}")
            if self.used + need > self.budget:
                self._retire_idle(need)
            if self.used + need > self.budget:
                return False
            st = _EngineState(self.engine_factory(job.model), job.model, need)
            self.engines[job.model.model_id] = st
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
        for shot in job.shots:
            st.queue.append((job, shot))
        job._left = len(job.shots)
        st.idle_since = None
        return True

    def _retire_idle(self, need):
        for mid, st in sorted(self.engines.items(), key=lambda kv: kv[1].idle_since or math.inf):
            if self.used + need <= self.budget:
                return
            if st.idle_since is not None and not st.queue and not st.running and not st.pending:
                st.engine.close()
                self.used -= st.footprint
                del self.engines[mid]

    def _fill(self, st):
        import torch
        while st.queue and len(st.running) < self.max_slots:
            job, shot = st.queue.popleft()
            shot.traces = torch.empty((shot.nt, shot.rec_xyz.shape[0]), dtype=torch.float32,
                                      device=shot.src_wav.device)
            slot = st.engine.add_shot(shot.nt, shot.src_xyz, shot.src_wav, shot.rec_xyz,
                                      shot.traces)
            st.running[slot] = (job, shot)

    def _advance(self, st):
        st.engine.step(self.chunk)
        finished = []
        for s, (job, shot) in st.running.items():
            if s not in st.finishing and st.engine.steps_left(s) == 0:
                st.finishing.add(s)
                finished.append((s, job, shot))
        st.pending.append((st.engine.record_event(), finished))

    def _deliver(self, st, now):
        keep = []
        for ev, items in st.pending:
            if ev.query():
                for s, job, shot in items:
                    cur = st.running.get(s)
                    if cur is None or cur[0] is not job or cur[1] is not shot:
                        continue
                    st.running.pop(s)
                    st.finishing.discard(s)
                    st.engine.release(s)
                    shot.done_at = now
                    if self.deliver is not None:
                        self.deliver(job, shot)
                    job._left -= 1
                    if job._left == 0:
                        job.done_at = now
                        self.jobs_done.append(job)
            else:
                keep.append((ev, items))
        st.pending = keep

    def run(self, jobs, idle_sleep=0.0005):
        """Serve `jobs` (each with an arrival time in seconds after the start)
        until all are done; returns the list of finished jobs."""
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        self.t0 = self.clock()
        total = len(jobs)
        while len(self.jobs_done) < total:
            now = self.clock() - self.t0
            while pending and pending[0].arrival <= now:
                self.waiting.append(pending.popleft())
            still = deque()
            while self.waiting:
                job = self.waiting.popleft()
                if not self._admit(job, now):
                    still.append(job)
            self.waiting = still
            busy = False
            inflight = 0
            for st in list(self.engines.values()):
                self._deliver(st, self.clock() - self.t0)
                self._fill(st)
                if st.running:
                    # keep at most two chunks in flight per engine
                    if len(st.pending) < 2:
                        self._advance(st)
                    busy = True
                    inflight += len(st.running)
                elif not st.queue and st.idle_since is None:
                    st.idle_since = now
            self.max_concurrent_shots = max(self.max_concurrent_shots, inflight)
            if not busy:
                if pending and not self.waiting:
                    time.sleep(max(0.0, min(idle_sleep * 20, pending[0].arrival - now)))
                else:
                    time.sleep(idle_sleep)
            else:
                time.sleep(idle_sleep)
        return self.jobs_done

    def close(self):
        for st in self.engines.values():
            st.engine.close()
        self.engines.clear()
        self.used = 0


# ---------------------------------------------------------------- baseline

def one_shot_per_launch(jobs, clock: Callable = time.perf_counter,
                        deliver: Optional[Callable] = None):
    """Every shot as its own acoustic_forward call, jobs in arrival order
    (single server).  Sets shot.traces / done_at and job.done_at, and calls
    deliver(job, shot) for every shot of a job once the job is done."""
    import torch
    t0 = clock()
    for job in sorted(jobs, key=lambda j: j.arrival):
        now = clock() - t0
        if now < job.arrival:
            time.sleep(job.arrival - now)
        md = job.model
        for shot in job.shots:
            rec, _ = acoustic_forward(md.grid, md.so, md.dt, shot.nt, md.m,
                                      shot.src_xyz[None].contiguous(),
                                      shot.src_wav[None].contiguous(),
                                      shot.rec_xyz[None].contiguous(), damp=md.damp,
                                      return_final=False)
            shot.traces = rec[0]
            shot.done_at = clock() - t0
        torch.cuda.synchronize()
        job.done_at = clock() - t0
        if deliver is not None:
            for shot in job.shots:
                deliver(job, shot)
    return jobs


def latency_stats(jobs):
    lat = np.array([j.latency for j in jobs if j.latency is not None])
    if lat.size == 0:
        return {}
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
