"""Benchmark of the acoustic FD sweep on GB300 (one JSON line on rank 0).

Workload (one benchmark "step"): the isotropic acoustic forward model on a
512^3 grid (h = 20 m, smooth-random velocity 1.5-4.5 km/s from seeded noise
with a 12-point Gaussian filter, 40-point absorbing border, one Ricker source,
512 x 512 receivers half a cell below the border, 1000 ms = 594 steps at the
CFL-limited dt) run once at each space order 4, 8, 12 and 16.  Metric:
grid-point updates per second (GPts/s) over the whole C-ABI calls, inputs
resident in HBM.  Every field is 512 MiB, larger than the 126 MB L2, so no L2
flush is needed between steps.

Also reported: the dominant kernel's roofline (acoustic_step, 16 algorithmic
bytes per point: read u^n, u^{n-1}, b; write u^{n+1}), the same metric end to
end with pinned host buffers (e2e), the FP64 CPU oracle on a bounded sample of
the workload (cpu_baseline), TTI throughput on the 512^3 TTI workload, SM
clocks sampled during the timed region and the number of kernel launches.

``--impl reference`` times the FP64 CPU oracle instead (the reference arm):
each step is one time step of the same 512^3 workload at each space order.

Multi-GPU (torchrun, one rank per GPU): shots are independent, so each rank
runs its own shot with no data-path collective (weak scaling); the timed
region is bracketed by barriers and the maximum over ranks is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

SO_LIST = (4, 8, 12, 16)
BYTES_PER_POINT_ACOUSTIC = 16.0  # read u^n, u^{n-1}, b; write u^{n+1}
BYTES_PER_POINT_STEP2 = 20.0     # two steps: read u^n, u^{n-1}, b; write u^{n+1}, u^{n+2}
ACOUSTIC_KERNELS = (("acoustic_step", BYTES_PER_POINT_ACOUSTIC, 1),
                    ("acoustic_step2", BYTES_PER_POINT_STEP2, 2))
BYTES_PER_POINT_TTI = 44.0       # p, r: read 2 levels + write 1 (24 B); m, eps, delta, theta, phi (20 B)
METRIC = "GPts/s (acoustic 512^3, so 4/8/12/16)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def _code_lines(text):
    """The lines of a source file without whole-line comments and blank lines
    (an edit of those does not change the kernel)."""
    return b"\n".join(l for l in text.split(b"\n")
                      if l.strip() and not l.lstrip().startswith(b"//"))


def kernel_source_hash():
    """Hash of the code the acoustic stencil kernels are built from (for
    kernels.cuh, only its acoustic section; whole-line comments left out), so
    that a recorded ncu traffic figure is reported only for the kernel
    version it was measured on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1807_03032_gb300", "csrc")
    for f in ("acoustic.cu", "acoustic2.cu", "f32x2.cuh", "common.cuh"):
        h.update(_code_lines(open(os.path.join(csrc, f), "rb").read()))
    k = open(os.path.join(csrc, "kernels.cuh"), "rb").read()
    a = k.find(b"// ---------------------------------------------------------------- acoustic K1")
    b = k.find(b"// ---------------------------------------------------------------- sparse K3/K4")
    h.update(_code_lines(k[a:b] if 0 <= a < b else k))
    return h.hexdigest()[:16]


def acoustic_kernel_stats(_native):
    """{family: (total ms, launches, points per launch)} of the acoustic
    stencil kernels from the library's statistics."""
    return {f: _native.stats_get(f) for f, _, _ in ACOUSTIC_KERNELS}


def roofline_of(family, st, peak, peak_kind, traffic=None):
    bpp = dict((f, b) for f, b, _ in ACOUSTIC_KERNELS)[family]
    ms, n, pts = st
    launch_ms = ms / max(n, 1)
    achieved = bpp * pts / (launch_ms * 1e-3) / 1e9 if n else 0.0
    return {"bound": "hbm", "kernel": family, "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4),
            "frac_of_nominal_8000": round(achieved / 8000.0, 4), "traffic": traffic,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback 6.8 TB/s",
            "bytes_per_point": bpp, "launch_ms": round(launch_ms, 4), "launches": int(n)}


def ncu_traffic():
    """Per-launch DRAM bytes of the acoustic kernels from the committed ncu
    summary ({family: {so: bytes}}), or None if the kernel sources changed
    since it was captured."""
    p = os.path.join(ROOT, "profiles", "acoustic_step_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_hash") != kernel_source_hash():
        return None
    return d


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            for name, v in zip(names, r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def shard_shots(nshots_total, rank, world):
    """Contiguous block of global shot indices owned by `rank` (shots are
    independent problems: no data moves between ranks)."""
    base, extra = divmod(nshots_total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value, world, device=None):
    """Maximum of a per-rank float over all ranks (the job's elapsed time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shot_source_offset(shot, spacing):
    """Global shot `shot` fires at the workload's source shifted 7 cells in x
    per shot index."""
    return np.float32(shot * 7 * spacing)


def build_workload(rank, n, so):
    w = workloads.acoustic_large(n=n, so=so, nt=None)
    shots = shard_shots(dist_env()[0], rank, dist_env()[0])
    w.src_xyz[..., 0] += shot_source_offset(shots[0], w.spacing[0])
    return w


def run_ours(args):
    import torch
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    _native.load()
    for so in args.so:
        if args.time_tiling == -1 or _native.num_time_tiling_configs(so) > 0:
            _native.set_time_tiling(so, args.time_tiling)

    n = args.n
    t0 = time.time()
    w = build_workload(rank, n, SO_LIST[0])
    log(f"[bench] workload built in {time.time() - t0:.1f}s: {w.name}, nt={w.nt}, dt={w.dt:.4f} ms")
    g = fd.Grid(w.shape, w.spacing, w.origin)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    m, damp, sxyz, swav, rxyz = T(w.m), T(w.damp), T(w.src_xyz), T(w.src_wav), T(w.rec_xyz)
    nrec = rxyz.shape[1]
    rec_out = torch.empty((1, w.nt, nrec), dtype=torch.float32, device=dev)
    points_per_forward = float(w.npoints) * (w.nt - 1) * w.nshots
    stream = torch.cuda.current_stream(dev)

    def step():
        for so in args.so:
            fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp,
                                rec_out=rec_out, return_final=False)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---------------------------------------------------------------- timed region
    _native.stats_reset()
    _native.stats_enable(True)
    launches0 = _native.launch_count()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    per_so_ms = {so: 0.0 for so in args.so}
    per_so_runs = {so: [] for so in args.so}  # one forward per benchmark step
    for _ in range(args.steps):
        for so in args.so:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp,
                                rec_out=rec_out, return_final=False)
            e1.record(stream)
            e1.synchronize()
            per_so_ms[so] += e0.elapsed_time(e1)
            per_so_runs[so].append(e0.elapsed_time(e1))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    launches = _native.launch_count() - launches0
    kst = acoustic_kernel_stats(_native)
    sp_ms, sp_n, _ = _native.stats_get("sparse")
    _native.stats_enable(False)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), ws, dev)
    total_points = points_per_forward * len(args.so) * args.steps * ws
    value = total_points / (elapsed_ms * 1e-3) / 1e9
    ms_per_step = elapsed_ms / args.steps

    # per space order: whole-call GPts/s and kernel roofline (per-so stats)
    per_so = {}
    for so in args.so:
        runs = sorted(per_so_runs[so])
        per_so[str(so)] = {
            "gpts": round(points_per_forward * args.steps / (per_so_ms[so] * 1e-3) / 1e9, 2),
            # the paper reports the best of three runs; min and median over the
            # timed steps are given alongside the mean
            "gpts_best": round(points_per_forward / (runs[0] * 1e-3) / 1e9, 2),
            "gpts_median": round(points_per_forward / (float(np.median(runs)) * 1e-3) / 1e9, 2)}
    peak, peak_kind = measured_peaks()
    # per space order: kernels, steps and algorithmic bytes (separate short
    # timed passes, one forward each)
    so_kernel = {}
    for so in args.so:
        _native.stats_reset()
        _native.stats_enable(True)
        fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp, rec_out=rec_out,
                            return_final=False)
        st = acoustic_kernel_stats(_native)
        _native.stats_enable(False)
        kms = sum(v[0] for v in st.values())
        steps = sum(st[f][1] * k for f, _, k in ACOUSTIC_KERNELS)
        pts_ = max(v[2] for v in st.values())
        alg = sum(b * st[f][1] * st[f][2] for f, b, _ in ACOUSTIC_KERNELS)
        main = max(st, key=lambda f: st[f][0])
        so_kernel[so] = main
        per_so[str(so)].update({
            "kernel": main, "kernel_gbs": round(alg / (kms * 1e-3) / 1e9, 1),
            "kernel_frac": round(alg / (kms * 1e-3) / 1e9 / peak, 4),
            "kernel_frac_of_nominal_8000": round(alg / (kms * 1e-3) / 1e9 / 8000.0, 4),
            "kernel_gpts": round(pts_ * steps / (kms * 1e-3) / 1e9, 2),
            "bytes_per_point_step": round(alg / (pts_ * steps), 2)})

    # roofline of the dominant kernel of the timed region (by device time),
    # and of every acoustic stencil kernel that ran
    tr = ncu_traffic()
    rooflines = {}
    for fam, _, _ in ACOUSTIC_KERNELS:
        if kst[fam][1] == 0:
            continue
        traffic = None
        if tr and fam in tr:
            sos = [so for so in args.so if so_kernel.get(so) == fam]
            vals = [tr[fam].get(str(so)) for so in sos]
            if sos and all(v is not None for v in vals):
                traffic = float(np.mean(vals)) * (kst[fam][2] / tr.get("points_per_launch",
                                                                        kst[fam][2]))
        rooflines[fam] = roofline_of(fam, kst[fam], peak, peak_kind, traffic)
    dominant = max(rooflines, key=lambda f: kst[f][0])
    roofline = dict(rooflines[dominant])
    roofline["sparse_launch_ms"] = round(sp_ms / max(sp_n, 1), 4)
    roofline["others"] = {f: r for f, r in rooflines.items() if f != dominant}

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hm, hdamp, hs, hw, hr = pin(w.m), pin(w.damp), pin(w.src_xyz), pin(w.src_wav), pin(w.rec_xyz)
        hrec = torch.empty((1, w.nt, nrec), dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * 4 for t in (hm, hdamp, hs, hw, hr)) * len(args.so)
        d2h = hrec.numel() * 4 * len(args.so)

        def step_host():
            for so in args.so:
                fd.acoustic_forward(g, so, w.dt, w.nt, hm, hs, hw, hr, damp=hdamp, rec_out=hrec,
                                    return_final=False, stream=stream.cuda_stream)

        step_host()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ksteps = max(1, min(args.steps, 3))
        for _ in range(ksteps):
            step_host()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        e_ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
        e2e = {"value": round(points_per_forward * len(args.so) * ksteps * ws / (e_ms * 1e-3) / 1e9, 2),
               "unit": "GPts/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": ksteps, "host_memory": "pinned"}

    # ---------------------------------------------------------------- binary16 storage
    storage_f16 = None
    if not args.no_f16:
        storage_f16 = run_storage_f16(args, fd, _native, g, w, m, damp, sxyz, swav, rxyz,
                                      stream, peak, per_so)

    # ---------------------------------------------------------------- 3-D damping field
    damp_field = None
    if not args.no_damp_field:
        damp_field = run_damp_field(args, fd, _native, g, w, m, damp, sxyz, swav, rxyz, stream,
                                    peak)

    # ---------------------------------------------------------------- TTI
    tti = None
    if not args.no_tti:
        del m, damp, sxyz, swav, rxyz, rec_out
        torch.cuda.empty_cache()
        tti = run_tti(args, fd, _native, dev, stream, peak)

    # ---------------------------------------------------------------- FWI gradient
    fwi = None
    if not args.no_fwi:
        torch.cuda.empty_cache()
        fwi = run_fwi(args, fd, dev, stream)

    # ---------------------------------------------------------------- serving
    serving = None
    if not args.no_serving and "8" in per_so:
        torch.cuda.empty_cache()
        serving = run_serving(args, fd, dev, per_so["8"]["kernel_gpts"])

    # ---------------------------------------------------------------- CPU baseline (oracle)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.so)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GPts/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"acoustic forward {n}^3, h=20 m, smooth-random v 1.5-4.5 km/s, "
                                   f"40-pt border, 1 Ricker source, {n}x{n} receivers, "
                                   f"nt={w.nt} (1000 ms), so in {list(args.so)}; one step = one "
                                   "forward per space order",
                       "grid": [n, n, n], "nt": w.nt, "so": list(args.so), "shots_per_gpu": 1,
                       "parallelism": f"shots x {ws} (replicas, no collective)",
                       "l2": "inputs larger than L2 (512 MiB per field); no flush",
                       "timing": "CUDA events on the calling stream around whole C-ABI calls; "
                                 "kernel times from the library's per-launch events"},
            "per_so": per_so,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "storage_f16": storage_f16,
            "damp_field": damp_field,
            "tti": tti,
            "fwi_gradient": fwi,
            "serving": serving,
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_storage_f16(args, fd, _native, g, w, m, damp, sxyz, swav, rxyz, stream, peak, per_so):
    """The same forward runs with the wavefields and b stored in binary16
    (FP32 arithmetic): whole-call and kernel rates, the kernel's HBM
    fraction at 8 algorithmic bytes per point, and the distance of its
    traces from the FP32 run's."""
    import torch
    nrec = rxyz.shape[1]
    rec32 = torch.empty((1, w.nt, nrec), dtype=torch.float32, device=m.device)
    rec16 = torch.empty_like(rec32)
    pts = float(w.npoints) * (w.nt - 1)
    out = {"what": "acoustic_forward_opts with FD_STORAGE_F16: u^n, u^{n-1} and b held in "
                   "IEEE binary16, FP32 arithmetic; one forward per so of the same workload",
           "bytes_per_point": 8, "per_so": {}}
    for so in args.so:
        fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp, rec_out=rec32,
                            return_final=False)
        fd.acoustic_forward(g, so, w.dt, 20, m, sxyz, swav[:, :20].contiguous(), rxyz,
                            damp=damp, return_final=False, storage="f16")
        _native.stats_reset()
        _native.stats_enable(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp, rec_out=rec16,
                            return_final=False, storage="f16")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, nl, npts = _native.stats_get("acoustic_step_h")
        _native.stats_enable(False)
        per = kms / max(nl, 1)
        gbs = 8.0 * npts / (per * 1e-3) / 1e9
        rel = float(torch.linalg.vector_norm((rec16 - rec32).double()) /
                    torch.linalg.vector_norm(rec32.double()))
        kg = npts / (per * 1e-3) / 1e9
        row = {"gpts": round(pts / (ms * 1e-3) / 1e9, 2), "kernel_gpts": round(kg, 2),
               "kernel_gbs": round(gbs, 1), "kernel_frac": round(gbs / peak, 4),
               "traces_rel_l2_vs_f32": float(f"{rel:.3e}")}
        k32 = per_so.get(str(so), {}).get("kernel_gpts")
        if k32:
            row["kernel_speedup_vs_f32"] = round(kg / k32, 3)
        out["per_so"][str(so)] = row
    return out


def run_damp_field(args, fd, _native, g, w, m, damp, sxyz, swav, rxyz, stream, peak):
    """The same forward runs with the damping given as a 3-D field (the
    workload's separable sponge expanded point by point; acoustic_forward_opts
    with FD_DAMP_FIELD): the stencil kernel then reads zeta = damp b / dt per
    point, 20 algorithmic bytes per point.  Kernel rate, its HBM fraction,
    and the distance of its traces from the profile path's."""
    import torch
    n = w.shape[0]
    dh = np.asarray(w.damp, dtype=np.float64)
    field = (dh[2 * n:, None, None] + dh[n:2 * n][None, :, None] + dh[:n][None, None, :])
    d3 = torch.from_numpy(np.ascontiguousarray(field, dtype=np.float32)).to(m.device)
    del field
    nrec = rxyz.shape[1]
    ra = torch.empty((1, w.nt, nrec), dtype=torch.float32, device=m.device)
    rf = torch.empty_like(ra)
    out = {"what": "acoustic_forward_opts with FD_DAMP_FIELD: the separable sponge given as a "
                   "3-D field; the kernel reads zeta = damp b / dt per point",
           "bytes_per_point": 20, "per_so": {}}
    for so in args.so:
        fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=damp, rec_out=ra,
                            return_final=False)
        _native.stats_reset()
        _native.stats_enable(True)
        fd.acoustic_forward(g, so, w.dt, w.nt, m, sxyz, swav, rxyz, damp=d3, rec_out=rf,
                            return_final=False, damp_layout="field")
        torch.cuda.synchronize()
        kms, nl, npts = _native.stats_get("acoustic_step")
        _native.stats_enable(False)
        per = kms / max(nl, 1)
        gbs = 20.0 * npts / (per * 1e-3) / 1e9
        rel = float(torch.linalg.vector_norm((rf - ra).double()) /
                    torch.linalg.vector_norm(ra.double()))
        out["per_so"][str(so)] = {"kernel_gpts": round(npts / (per * 1e-3) / 1e9, 2),
                                  "kernel_gbs": round(gbs, 1), "kernel_frac": round(gbs / peak, 4),
                                  "traces_rel_l2_vs_profiles": float(f"{rel:.3e}")}
    del d3
    torch.cuda.empty_cache()
    return out


def run_tti(args, fd, _native, dev, stream, peak):
    import torch
    n = args.n
    t0 = time.time()
    w = workloads.tti_large(n=n, so=4)
    log(f"[bench] TTI workload built in {time.time() - t0:.1f}s, nt={w.nt}")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    arrs = [T(a) for a in (w.m, w.eps, w.delta, w.theta, w.phi, w.src_xyz, w.src_wav, w.rec_xyz,
                           w.damp)]
    m, e, d, th, ph, sx, sw, rx, dd = arrs
    rec = torch.empty((1, w.nt, rx.shape[1]), dtype=torch.float32, device=dev)
    out = {"workload": f"TTI {n}^3 two-layer 1.5/2.5 km/s, eps U[0,0.3], delta U[0,0.2] "
                       f"(<= eps), theta/phi smooth in [0, pi/4], nt={w.nt}",
           "bytes_per_point": BYTES_PER_POINT_TTI, "per_so": {}}
    pts = float(w.npoints) * (w.nt - 1)
    for so in args.so:
        fd.tti_forward(g, so, w.dt, 20, m, e, d, th, ph, sx, sw[:, :20].contiguous(), rx,
                       damp=dd, rec_out=rec[:, :20].contiguous(), return_final=False)
        _native.stats_reset()
        _native.stats_enable(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fd.tti_forward(g, so, w.dt, w.nt, m, e, d, th, ph, sx, sw, rx, damp=dd, rec_out=rec,
                       return_final=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        p1 = _native.stats_get("tti_pass1")
        p2 = _native.stats_get("tti_pass2")
        pf = _native.stats_get("tti_fused")
        _native.stats_enable(False)
        steps = max(p1[1], pf[1], 1)
        kms = (p1[0] + p2[0] + pf[0]) / steps
        npts = max(p1[2], pf[2])
        gb = BYTES_PER_POINT_TTI * npts / (kms * 1e-3) / 1e9
        row = {"gpts": round(pts / (ms * 1e-3) / 1e9, 2), "step_kernel_ms": round(kms, 4),
               "kernel_gpts": round(npts / (kms * 1e-3) / 1e9, 2),
               "scheme": "fused" if pf[1] else "two_pass", "hbm_frac_44B": round(gb / peak, 4)}
        if p1[1]:
            row.update({"pass1_ms": round(p1[0] / p1[1], 4), "pass2_ms": round(p2[0] / p2[1], 4)})
        out["per_so"][str(so)] = row
    if not args.no_tti_ablation:
        out["ablation"] = run_tti_ablation(args, fd, _native, g, w, m, e, d, th, ph, sx, sw, rx,
                                           dd, out["per_so"])
    return out


def run_tti_ablation(args, fd, _native, g, w, m, e, d, th, ph, sx, sw, rx, dd, per_so):
    """TTI variants on the same workload, per-step kernel time over a short
    run: temporaries in HBM (two passes), temporaries in shared memory (one
    fused pass, so <= 8) and recomputed inner derivatives (one pass), centred
    vs staggered first derivatives.  FMA counts per point per step
    are those of the kernel sources (R = so/2): two passes 24R + 30, recompute
    72R^2 + 60R (the inner gradient of p and r at each of the 6R outer taps)."""
    import torch
    nt_ab = 24
    sw_ab = sw[:, :nt_ab].contiguous()
    rec = torch.empty((1, nt_ab, rx.shape[1]), dtype=torch.float32, device=sw.device)
    res = {"steps": nt_ab - 1, "note": "per-step kernel ms from the library's per-launch events; "
           "two_pass_centred from the main TTI run"}
    for so in args.so:
        R = so // 2
        row = {"fma_per_point": {"two_pass": 24 * R + 30, "recompute": 72 * R * R + 60 * R}}
        if per_so[str(so)]["scheme"] == "two_pass":
            row["two_pass_centred_ms"] = per_so[str(so)]["step_kernel_ms"]
        variants = [("staggered", "two_pass", "two_pass_staggered_ms"),
                    ("centred", "recompute", "recompute_centred_ms"),
                    ("staggered", "recompute", "recompute_staggered_ms")]
        if "two_pass_centred_ms" not in row:
            variants.insert(0, ("centred", "two_pass", "two_pass_centred_ms"))
        if so <= 8:  # temporaries in shared memory: radii up to 4
            variants.append(("centred", "fused", "fused_centred_ms"))
        for deriv, scheme, key in variants:
            fd.tti_forward(g, so, w.dt, 4, m, e, d, th, ph, sx, sw_ab[:, :4].contiguous(), rx,
                           damp=dd, rec_out=rec[:, :4].contiguous(), return_final=False,
                           deriv=deriv, scheme=scheme)
            _native.stats_reset()
            _native.stats_enable(True)
            fd.tti_forward(g, so, w.dt, nt_ab, m, e, d, th, ph, sx, sw_ab, rx, damp=dd,
                           rec_out=rec, return_final=False, deriv=deriv, scheme=scheme)
            torch.cuda.synchronize()
            if scheme == "two_pass":
                p1 = _native.stats_get("tti_pass1")
                p2 = _native.stats_get("tti_pass2")
                kms = (p1[0] + p2[0]) / max(p1[1], 1)
            else:
                pr = _native.stats_get("tti_" + scheme)
                kms = pr[0] / max(pr[1], 1)
            _native.stats_enable(False)
            row[key] = round(kms, 4)
        row["recompute_over_two_pass"] = round(row["recompute_centred_ms"] /
                                               row["two_pass_centred_ms"], 2)
        if "fused_centred_ms" in row:
            row["fused_over_two_pass"] = round(row["fused_centred_ms"] /
                                               row["two_pass_centred_ms"], 2)
        res[str(so)] = row
        log(f"[bench] TTI ablation so={so}: {row}")
    return res


def run_fwi(args, fd, dev, stream):
    """FWI gradient on the 256^3 layered model: 16 shots, 256 x 256 receivers,
    so = 8, nt = 2000, checkpoint every 45 steps.  Timed: the forward model of
    all shots in the initial model, the residual, and the checkpointed
    adjoint-state gradient."""
    import torch
    n, nt, nshots, K = args.fwi_n, args.fwi_nt, 16, 45
    t0 = time.time()
    true, init = workloads.fwi_layered(n=n, so=8, nt=nt, nshots=nshots)
    log(f"[bench] FWI workload built in {time.time() - t0:.1f}s")
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    g = fd.Grid(init.shape, init.spacing, init.origin)
    mt, m0, damp, sx, sw, rx = (T(a) for a in (true.m, init.m, init.damp, init.src_xyz,
                                               init.src_wav, init.rec_xyz))
    dobs, _ = fd.acoustic_forward(g, 8, init.dt, nt, mt, sx, sw, rx, damp=damp,
                                  return_final=False)
    # warm-up on a short window
    fd.acoustic_gradient(g, 8, init.dt, 40, m0, sx[:1], sw[:1, :40].contiguous(), rx[:1],
                         dobs[:1, :40].contiguous(), damp=damp, checkpoint_every=7)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    dpred, _ = fd.acoustic_forward(g, 8, init.dt, nt, m0, sx, sw, rx, damp=damp,
                                   return_final=False)
    resid = dpred - dobs
    e1.record(stream)
    grad = fd.acoustic_gradient(g, 8, init.dt, nt, m0, sx, sw, rx, resid, damp=damp,
                                checkpoint_every=K)
    e2.record(stream)
    torch.cuda.synchronize()
    fwd_ms, grad_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    pts = float(init.npoints) * (nt - 1) * nshots
    ok = bool(torch.isfinite(grad).all())
    return {"workload": f"FWI gradient {n}^3 layered 1.5-3.5 km/s (initial = true smoothed "
                        f"sigma 10), so 8, nt {nt}, {nshots} shots, {n}x{n} receivers, "
                        f"checkpoint every {K}",
            "forward_gpts": round(pts / (fwd_ms * 1e-3) / 1e9, 2),
            "gradient_gpts": round(pts / (grad_ms * 1e-3) / 1e9, 2),
            "gradient_s": round(grad_ms * 1e-3, 3), "forward_s": round(fwd_ms * 1e-3, 3),
            "objective": float(0.5 * (resid.double() ** 2).sum()), "finite": ok,
            "note": "gradient GPts/s counts forward-model grid-point updates (nt-1 per shot); "
                    "the gradient performs a forward with checkpoints, a recomputation and "
                    "an adjoint sweep",
            "parity": "tests/test_gpu_fwi_scale.py: the same recipe at 96^3, 4 shots in 2 "
                      "batches, nt 400, checkpoint every 20: GPU gradient vs the FP64 oracle "
                      "gradient within 1e-4 (relative L2 and max-abs), and Taylor slopes 1 and 2 "
                      "of the GPU objective with the GPU gradient"}


def serving_jobs(fd, dev, rate_jobs_per_s, n_jobs, seed=6, sizes=(128, 256, 384), h=20.0,
                 nt_range=(500, 3000), shots_range=(1, 32), so=8, nbl=20):
    """Served shot stream: Poisson arrivals (seeded) of jobs on one model per
    grid size in {128^3, 256^3, 384^3} (uniform), nt ~ U{500..3000},
    1..32 shots per job, so = 8, 128 x 128 receivers at a stride of N/128."""
    import torch
    from paper_1807_03032_gb300.serving import Job, Model, Shot
    rng = np.random.default_rng(seed)
    models = {}
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    for i, n in enumerate(sizes):
        shape = (n, n, n)
        v = workloads.two_layer_velocity(shape, 1.5, 3.0 + 0.25 * i, interface=n // 2)
        dt = workloads.cfl_dt((h, h, h), 3.0 + 0.25 * i)
        models[n] = Model(i, fd.Grid(shape, (h, h, h)), so, dt,
                          T(workloads.slowness_squared(v)),
                          T(workloads.damping_profile(shape, nbl, (h, h, h), 3.0 + 0.25 * i)))
    jobs, t = [], 0.0
    for j in range(n_jobs):
        t += rng.exponential(1.0 / rate_jobs_per_s)
        n = int(rng.choice(sizes))
        md = models[n]
        stride = n // 128
        gy, gx = np.meshgrid(np.arange(0, n, stride) * h, np.arange(0, n, stride) * h,
                             indexing="ij")
        rec = np.stack([gx.ravel(), gy.ravel(), np.full(gx.size, nbl * h + 0.5 * h)], -1)
        rec_t = T(rec.astype(np.float32))
        shots = []
        for _ in range(int(rng.integers(shots_range[0], shots_range[1] + 1))):
            nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
            src = np.array([[rng.uniform(nbl, n - 1 - nbl) * h, rng.uniform(nbl, n - 1 - nbl) * h,
                             nbl * h + 20.0]], np.float32)
            wav = workloads.ricker(nt, md.dt)[:, None].astype(np.float32)
            shots.append(Shot(nt, T(src), T(wav), rec_t))
        jobs.append(Job(j, md, shots, t))
    return jobs


def run_serving(args, fd, dev, gpts_so8):
    """Continuous-batching server vs one acoustic_forward call per shot, same
    arrivals; rate = 0.8 x the capacity implied by the measured so-8 kernel
    throughput of this run."""
    import torch
    from paper_1807_03032_gb300.serving import Server, checksum_and_drop, latency_stats, \
        one_shot_per_launch
    sizes = (128, 256, 384)
    mean_pts = np.mean([n ** 3 for n in sizes]) * 1750.0 * 16.5
    capacity = gpts_so8 * 1e9 / mean_pts
    rate = 0.8 * capacity
    jobs = serving_jobs(fd, dev, rate, args.serve_jobs)
    nshots = sum(len(j.shots) for j in jobs)
    pts = sum(j.model.grid.shape[0] ** 3 * (s.nt - 1) for j in jobs for s in j.shots)
    srv = Server(hbm_budget=int(args.serve_budget_gb * (1 << 30)), max_slots=32, chunk=32,
                 max_nsrc=1, max_nrec=128 * 128, deliver=checksum_and_drop)
    t0 = time.perf_counter()
    srv.run(jobs)
    make = time.perf_counter() - t0
    srv.close()
    served = {"shots_per_s": round(nshots / make, 3), "gpts": round(pts / make / 1e9, 2),
              "makespan_s": round(make, 2), **{k: round(v, 3) for k, v in latency_stats(jobs).items()},
              "max_concurrent_shots": srv.max_concurrent_shots,
              "peak_engine_bytes": srv.peak_used}
    for j in jobs:
        for s in j.shots:
            s.traces = None
        j.done_at = None
    torch.cuda.empty_cache()
    sums = [s.checksum for j in jobs for s in j.shots]
    t0 = time.perf_counter()
    one_shot_per_launch(jobs, deliver=checksum_and_drop)
    make_b = time.perf_counter() - t0
    # the same traces from both paths (sums of squares, relative)
    agree = max(abs(float(a) - float(s.checksum)) / max(float(s.checksum), 1e-300)
                for a, s in zip(sums, (s for j in jobs for s in j.shots)))
    base = {"shots_per_s": round(nshots / make_b, 3), "gpts": round(pts / make_b / 1e9, 2),
            "makespan_s": round(make_b, 2), **{k: round(v, 3) for k, v in latency_stats(jobs).items()}}
    return {"workload": f"{len(jobs)} jobs / {nshots} shots, Poisson arrivals at "
                        f"{rate:.3f} jobs/s (0.8 x capacity {capacity:.3f} from the so-8 kernel "
                        f"rate {gpts_so8:.0f} GPts/s), grids {{128,256,384}}^3, nt U{{500..3000}}, "
                        f"1-32 shots per job, so 8, 128x128 receivers",
            "batched": served, "one_shot_per_launch": base,
            "traces_sum_of_squares_max_rel_diff": float(f"{agree:.3e}"),
            "latency_is": "job arrival to delivery of its last shot's traces (device)"}


def run_serving_only(args):
    """The served shot stream alone (config: Poisson arrivals, grids {128, 256,
    384}^3, nt U{500..3000}, 1-32 shots per job, so 8), batched server against
    one acoustic_forward call per shot, with `--serve-jobs` jobs so that p99
    is a tail and not the maximum.  The arrival rate is 0.8 x the capacity
    implied by the so-8 kernel rate measured here on a 512^3 forward."""
    import torch
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    dev = torch.device("cuda", 0)
    w = workloads.acoustic_large(n=512, so=8, nt=40)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    m, damp, sx, sw, rx = T(w.m), T(w.damp), T(w.src_xyz), T(w.src_wav), T(w.rec_xyz)
    fd.acoustic_forward(g, 8, w.dt, w.nt, m, sx, sw, rx, damp=damp, return_final=False)
    _native.stats_reset()
    _native.stats_enable(True)
    fd.acoustic_forward(g, 8, w.dt, w.nt, m, sx, sw, rx, damp=damp, return_final=False)
    torch.cuda.synchronize()
    ms, k, pts = _native.stats_get("acoustic_step")
    _native.stats_enable(False)
    gpts = pts / (ms / k * 1e-3) / 1e9
    del m, damp, sx, sw, rx
    torch.cuda.empty_cache()
    out = run_serving(args, fd, dev, gpts)
    print(json.dumps({"serving": out}), flush=True)


def run_batched_probe(args):
    """Diagnostic (not the benchmark line): one forward of S shots sharing a
    two-layer n^3 model (acoustic, or TTI with the benchmark's anisotropy
    recipe; space order --batched-so, nt 4, one source and one receiver per
    shot), then three 12-step calls timed with the library's per-launch
    events; prints the stencil kernels' time per step and rate over all
    shots.  Used to capture the DRAM bytes per shot-point of a shot-batched
    launch with ncu."""
    import torch
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    S, n, h, so = args.batched_probe, args.batched_n, 20.0, args.batched_so
    tti = args.batched_kind == "tti"
    shape = (n, n, n)
    m = workloads.slowness_squared(workloads.two_layer_velocity(shape, 1.5, 2.5))
    damp = workloads.damping_profile(shape, 20, (h, h, h), 2.5)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    if tti:
        aniso = [T(f) for f in workloads.tti_fields(shape)]
        dt = workloads.cfl_dt((h, h, h), 2.5, eps_max=float(aniso[0].max()))
        fams = ("tti_pass1", "tti_pass2", "tti_fused")
    else:
        dt = workloads.cfl_dt((h, h, h), 2.5)
        fams = ("acoustic_step",)
    c = (n / 2 - 0.5) * h
    g = fd.Grid(shape, (h, h, h))
    mt, dd = T(m), T(damp)
    sx = T(np.tile(np.array([c, c, 30 * h]), (S, 1, 1)))
    rx = T(np.tile(np.array([[c, c, 25 * h]]), (S, 1, 1)))
    for i, nt in enumerate((4, 12, 12, 12)):
        if i == 1:
            torch.cuda.synchronize()
            _native.stats_reset()
            _native.stats_enable(True)
        sw = T(np.tile(workloads.ricker(nt, dt)[None, :, None], (S, 1, 1)))
        if tti:
            fd.tti_forward(g, so, dt, nt, mt, *aniso, sx, sw, rx, damp=dd, return_final=False)
        else:
            fd.acoustic_forward(g, so, dt, nt, mt, sx, sw, rx, damp=dd, return_final=False)
    torch.cuda.synchronize()
    st = [_native.stats_get(f) for f in fams]
    _native.stats_enable(False)
    steps = max(k for _, k, _ in st)
    ms = sum(t for t, _, _ in st) / steps
    pts = max(p for _, _, p in st)
    print(json.dumps({"probe": "batched shots", "kind": args.batched_kind, "shots": S,
                      "grid": n, "so": so, "kernel_us_per_step": round(ms * 1e3, 1),
                      "kernel_gpts_all_shots": round(pts / (ms * 1e-3) / 1e9, 1)}), flush=True)


def cpu_baseline(w, so_list):
    """The FP64 oracle, as it stands, on the host cores: one time step of the
    512^3 workload at each space order (a bounded sample of the workload)."""
    import oracle
    g = oracle.make_grid(w.shape, w.spacing, w.origin)
    cores = os.cpu_count() or 1
    t_total = 0.0
    pts = 0.0
    per_so = {}
    for so in so_list:
        t0 = time.perf_counter()
        oracle.acoustic_forward(g, so, w.dt, 2, w.m, w.src_xyz, w.src_wav[:, :2], w.rec_xyz,
                                damp=w.damp)
        dt_so = time.perf_counter() - t0
        t_total += dt_so
        pts += float(w.npoints)
        per_so[str(so)] = round(float(w.npoints) / dt_so / 1e9, 4)
    out = {"value": round(pts / t_total / 1e9, 4), "unit": "GPts/s", "cores": cores,
           "kind": "oracle",
           "sample": f"1 time step at each so in {list(so_list)} of the {w.shape[0]}^3 workload "
                     "(FP64 C oracle, OpenMP over all host cores, setup included)",
           "seconds": round(t_total, 2), "per_so": per_so}
    # the same oracle on one core, on a 256^3 sample of the workload recipe
    code = ("import json, time, oracle, workloads\n"
            "w = workloads.acoustic_large(n=256, so=4)\n"
            "g = oracle.make_grid(w.shape, w.spacing, w.origin)\n"
            "t = 0.0\n"
            f"for so in {list(so_list)}:\n"
            "    t0 = time.perf_counter()\n"
            "    oracle.acoustic_forward(g, so, w.dt, 2, w.m, w.src_xyz, w.src_wav[:, :2], "
            "w.rec_xyz, damp=w.damp)\n"
            "    t += time.perf_counter() - t0\n"
            f"print(json.dumps({{'seconds': t, 'points': float(w.npoints) * {len(so_list)}}}))\n")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                           env={**os.environ, "OMP_NUM_THREADS": "1"}, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": round(d["points"] / d["seconds"] / 1e9, 5),
                                "unit": "GPts/s", "cores": 1, "seconds": round(d["seconds"], 2),
                                "sample": f"1 time step at each so in {list(so_list)} of the "
                                          "256^3 version of the workload"}
    except Exception as exc:  # the single-core figure is informative only
        out["single_thread"] = {"error": str(exc)[:200]}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = args.n
    w = build_workload(0, n, SO_LIST[0])
    g = oracle.make_grid(w.shape, w.spacing, w.origin)
    cores = os.cpu_count() or 1

    def step():
        for so in args.so:
            oracle.acoustic_forward(g, so, w.dt, 2, w.m, w.src_xyz, w.src_wav[:, :2], w.rec_xyz,
                                    damp=w.damp)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = time.perf_counter() - t0
    pts = float(w.npoints) * len(args.so) * args.steps
    value = pts / t / 1e9
    sample = (f"each step = 1 time step of the {n}^3 acoustic workload at each so in "
              f"{list(args.so)} (FP64 C oracle, OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GPts/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"acoustic forward {n}^3, so in {list(args.so)}, sample of "
                                   "the GPU arm's workload", "grid": [n, n, n]},
            "cpu_baseline": {"value": round(value, 4), "unit": "GPts/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GPts/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--so", type=int, nargs="+", default=list(SO_LIST))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tti", action="store_true")
    ap.add_argument("--no-tti-ablation", action="store_true")
    ap.add_argument("--no-f16", action="store_true",
                    help="skip the binary16-storage runs")
    ap.add_argument("--time-tiling", type=int, default=-1,
                    help="fd_set_time_tiling mode for every space order (-1 automatic, "
                         "0 off, 1 + k two-step kernel configuration k)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-damp-field", action="store_true",
                    help="skip the 3-D damping-field runs")
    ap.add_argument("--no-fwi", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=10)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--fwi-n", type=int, default=256)
    ap.add_argument("--fwi-nt", type=int, default=2000)
    ap.add_argument("--batched-probe", type=int, default=0, metavar="S",
                    help="diagnostic only: one forward of S shots on a 256^3 model")
    ap.add_argument("--batched-n", type=int, default=256)
    ap.add_argument("--batched-so", type=int, default=8)
    ap.add_argument("--batched-kind", choices=("acoustic", "tti"), default="acoustic")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the served shot stream (with --serve-jobs jobs)")
    args = ap.parse_args()
    args.so = tuple(args.so)
    if args.batched_probe:
        run_batched_probe(args)
    elif args.serving_only:
        run_serving_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
