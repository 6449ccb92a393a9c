"""The multi-GPU path on CPU ranks (gloo, world size 2).

Shots are independent problems, so the benchmark shards them over ranks with
no data-path collective and reduces only the elapsed time (max over ranks).
Here two gloo ranks run their shards of a 4-shot problem through the oracle,
gather the traces, and rank 0 checks they equal the single-process run; the
time reduction and the shard arithmetic are checked too.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    w = workloads.acoustic_small(so=4, nt=12)
    nshots = 4
    src = np.concatenate([w.src_xyz.copy() for _ in range(nshots)], 0)
    for s in range(nshots):
        src[s, :, 0] += bench.shot_source_offset(s, w.spacing[0])
    wav = np.concatenate([w.src_wav] * nshots, 0)
    rec = np.concatenate([w.rec_xyz] * nshots, 0)
    return w, src, wav, rec


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, src, wav, rec = _problem()
        shots = bench.shard_shots(src.shape[0], rank, world)
        g = oracle.make_grid(w.shape, w.spacing, w.origin)
        r, _ = oracle.acoustic_forward(g, w.so, w.dt, w.nt, w.m, src[shots.start:shots.stop],
                                       wav[shots.start:shots.stop], rec[shots.start:shots.stop],
                                       damp=w.damp)
        gathered = [None] * world
        dist.all_gather_object(gathered, (shots.start, r))
        t = bench.max_over_ranks(10.0 + rank, world)
        if rank == 0:
            full = np.concatenate([g_[1] for g_ in sorted(gathered, key=lambda x: x[0])], 0)
            np.save(out_path, full)
            assert t == 10.0 + world - 1
    finally:
        dist.destroy_process_group()


def test_shard_arithmetic():
    for total in (1, 2, 5, 8, 13):
        for world in (1, 2, 3, 8):
            parts = [bench.shard_shots(total, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(total))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_two_gloo_ranks_equal_single_process(tmp_path):
    out = str(tmp_path / "traces.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    w, src, wav, rec = _problem()
    g = oracle.make_grid(w.shape, w.spacing, w.origin)
    ref, _ = oracle.acoustic_forward(g, w.so, w.dt, w.nt, w.m, src, wav, rec, damp=w.damp)
    got = np.load(out)
    np.testing.assert_array_equal(got, ref)
