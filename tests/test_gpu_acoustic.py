"""GPU parity of the acoustic forward path (K0 setup, K1 stencil, K3/K4 sparse,
graph-captured time loop) against the FP64 oracle, through the C ABI."""
import functools
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, max_abs_rel, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def long_run_trace_norm(so):
    w = workloads.acoustic_small(so=so, nt=400)
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    rref, _ = oracle.acoustic_forward(og, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                      w.rec_xyz, damp=w.damp)
    return float(np.linalg.norm(rref))


def run_pair(w, damp=True, u_init=None, host=False):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    g = fd.Grid(w.shape, w.spacing, w.origin)
    d = w.damp if damp else None
    if host:
        rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav, w.rec_xyz,
                                      damp=d, u_init=u_init)
    else:
        m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, d, u_init)
        rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
        torch.cuda.synchronize()
        rec, uf = rec.cpu().numpy(), uf.cpu().numpy()
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    rref, uref = oracle.acoustic_forward(og, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                         w.rec_xyz, damp=d, u_init=u_init)
    return rec, uf, rref, uref


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_small_config_parity(so):
    """64^3 two-layer model, 10-point border, so 4..16, nt = 100."""
    w = workloads.acoustic_small(so=so, nt=100)
    rec, uf, rref, uref = run_pair(w)
    assert rel_l2(uf, uref) <= TOL
    # By t = 150 ms only the wavelet's precursor has reached the receivers:
    # compare the traces against a floor of 1e-3 times the trace norm of the
    # nt = 400 run, in which the direct and reflected waves arrive.
    floor = 1e-3 * long_run_trace_norm(so)
    assert rel_l2(rec, rref, floor=floor) <= TOL
    assert np.all(np.isfinite(uf))


@pytest.mark.parametrize("so", [4, 16])
def test_small_config_long_run_traces(so):
    """nt = 400: the direct and reflected waves reach the receiver line."""
    w = workloads.acoustic_small(so=so, nt=400)
    rec, uf, rref, uref = run_pair(w)
    assert np.linalg.norm(rref) > 1e-3
    assert rel_l2(rec, rref) <= TOL
    assert rel_l2(uf, uref) <= TOL


def ragged_problem(so, nshots=2, nt=37, seed=3):
    """Ragged box (nx not a multiple of 4, partial tiles in x and y, odd nz),
    anisotropic spacing, shifted origin, several shots, colliding sources,
    random initial state."""
    shape = (31, 23, 45)  # nz, ny, nx
    h = (9.0, 11.0, 10.0)
    o = (-100.0, 250.0, 30.0)
    rng = np.random.default_rng(seed)
    v = 1.5 + 2.0 * workloads.smooth_random(shape, seed, 3.0, 0.0, 1.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 5, h, 3.5)
    dt = 0.9 * workloads.cfl_dt(h, 3.5)
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    nsrc, nrec = 3, 17
    src = o + rng.uniform(0.05, 0.95, (nshots, nsrc, 3)) * ext
    src[:, 1] = src[:, 0]  # two sources on the same point
    rec = o + rng.uniform(0.0, 1.0, (nshots, nrec, 3)) * ext
    rec[:, 0] = o + ext       # last node in every axis
    rec[:, 1] = o             # origin
    wav = rng.standard_normal((nshots, nt, nsrc))
    u_init = 1e-2 * workloads.random_wavefields(shape, seed, nshots=nshots, sigma=2.0)
    return workloads.Workload("ragged", shape, h, o, so, dt, nt, m, damp,
                              src.astype(np.float32), wav.astype(np.float32),
                              rec.astype(np.float32)), u_init


def separate_sources(w):
    """Moves the sources cells apart: no two injections share a node, so the
    order of the atomic additions cannot change a bit."""
    ext = np.array([(w.shape[2] - 1) * w.spacing[0], (w.shape[1] - 1) * w.spacing[1],
                    (w.shape[0] - 1) * w.spacing[2]])
    for k, f in enumerate((0.2, 0.5, 0.8)[:w.src_xyz.shape[1]]):
        w.src_xyz[:, k] = (np.asarray(w.origin) + f * ext).astype(np.float32)


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_ragged_multishot_parity(so):
    w, u_init = ragged_problem(so)
    rec, uf, rref, uref = run_pair(w, u_init=u_init)
    assert rel_l2(uf, uref) <= TOL
    assert rel_l2(rec, rref) <= TOL
    for s in range(w.nshots):
        assert rel_l2(uf[s], uref[s]) <= TOL


def test_host_buffers_match_device_buffers():
    w, u_init = ragged_problem(8, nshots=1, nt=20)
    separate_sources(w)
    torch = require_cuda()
    rec_h, uf_h, rref, uref = run_pair(w, u_init=u_init, host=True)
    rec_d, uf_d, _, _ = run_pair(w, u_init=u_init, host=False)
    np.testing.assert_array_equal(uf_h, uf_d)
    np.testing.assert_array_equal(rec_h, rec_d)
    assert rel_l2(uf_h, uref) <= TOL
    del torch


@pytest.mark.parametrize("nt", [70, 71])
def test_host_traces_streamed_during_graph_loop(nt):
    """Host receiver buffers are filled chunk by chunk while the graph-replayed
    time loop runs; the result equals the device-buffer run."""
    w, u_init = ragged_problem(8, nshots=2, nt=nt)
    separate_sources(w)
    torch = require_cuda()
    rec_h, uf_h, rref, uref = run_pair(w, u_init=u_init, host=True)
    rec_d, uf_d, _, _ = run_pair(w, u_init=u_init, host=False)
    np.testing.assert_array_equal(rec_h, rec_d)
    np.testing.assert_array_equal(uf_h, uf_d)
    assert rel_l2(rec_h, rref) <= TOL
    del torch


def test_no_steps_no_sparse_points():
    """nt = 1 (no step): the final state is the initial state and the single
    trace sample interpolates it; nsrc = nrec = 0 is accepted."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w, u_init = ragged_problem(4, nshots=1, nt=1)
    rec, uf, rref, uref = run_pair(w, u_init=u_init)
    np.testing.assert_array_equal(uf, u_init)
    assert rel_l2(rec, rref) <= 1e-6
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, = to_dev(torch, w.m)
    empty = torch.zeros((1, 0, 3), device="cuda")
    rec2, uf2 = fd.acoustic_forward(g, 4, w.dt, 5, m, empty, torch.zeros((1, 5, 0), device="cuda"),
                                    empty)
    assert rec2.shape == (1, 5, 0)
    assert float(uf2.abs().max()) == 0.0


def test_all_tile_configs_agree_bitwise_and_runs_are_deterministic():
    """Every compiled tile shape evaluates each point with the same operation
    order, so all configurations give bit-identical results; a repeated run
    is bit-identical too (sources on distinct nodes)."""
    require_cuda()
    from paper_1807_03032_gb300 import _native
    for so in (2, 4, 8, 12, 16):
        w, u_init = ragged_problem(so, nshots=1, nt=12)
        separate_sources(w)
        outs = []
        try:
            for cfg in range(_native.num_acoustic_configs(so)):
                _native.set_acoustic_config(so, cfg)
                outs.append(_gpu_only(w, u_init))
            again = _gpu_only(w, u_init)
        finally:
            _native.set_acoustic_config(so, -1)
        for rec, uf in outs[1:] + [again]:
            np.testing.assert_array_equal(uf, outs[0][1])
            np.testing.assert_array_equal(rec, outs[0][0])


def _gpu_only(w, u_init):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp, u_init)
    rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
    torch.cuda.synchronize()
    return rec.cpu().numpy(), uf.cpu().numpy()


def test_graph_path_equals_direct_launches():
    """Statistics mode launches every step directly; the default path replays
    a captured graph.  Both must give identical results (nt > 2 chunks)."""
    from paper_1807_03032_gb300 import _native
    w, u_init = ragged_problem(8, nshots=1, nt=70)
    a = _gpu_only(w, u_init)
    _native.stats_enable(True)
    try:
        b = _gpu_only(w, u_init)
    finally:
        _native.stats_enable(False)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    ms, n, pts = _native.stats_get("acoustic_step")
    assert n >= 69 and ms > 0 and pts == float(np.prod(w.shape))


def test_errors_are_reported():
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import FdError
    w = workloads.acoustic_small(so=4, nt=10)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz)
    # dt above the stability bound (bound = 0.5 h / v_max for so = 4)
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, 0.51 * 10.0 / 2.5, 10, m, sx, sw, rx)
    assert e.value.name == "FD_ERR_CFL"
    fd.acoustic_forward(g, 4, 0.49 * 10.0 / 2.5, 10, m, sx, sw, rx)
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 6, w.dt, 10, m, sx, sw, rx)
    assert e.value.name == "FD_ERR_SO"
    bad = rx.clone()
    bad[0, 3, 2] = 64 * 10.0  # one cell beyond the last node
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, w.dt, 10, m, sx, sw, bad)
    assert e.value.name == "FD_ERR_COORD"
    m2 = m.clone()
    m2[3, 4, 5] = -1.0
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, w.dt, 10, m2, sx, sw, rx)
    assert e.value.name == "FD_ERR_ARG"
    m2[3, 4, 5] = float("nan")
    with pytest.raises(FdError) as e:
        fd.acoustic_forward(g, 4, w.dt, 10, m2, sx, sw, rx)
    assert e.value.name == "FD_ERR_ARG"
    # the library still works after the errors
    rec, _ = fd.acoustic_forward(g, 4, w.dt, 10, m, sx, sw, rx)
    assert torch.isfinite(rec).all()


def test_full_size_parity_first_steps():
    """512^3 (the benchmark's grid and launch configuration), so = 4, 8, 12
    and 16: four steps from a smooth random state with a source (injected by
    the stencil kernel) and the full 512 x 512 receiver plane, against the
    oracle at every point."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    n = 512
    for so in (4, 8, 12, 16):
        w = workloads.acoustic_large(n=n, so=so, nt=4)
        u_init = 0.01 * workloads.random_wavefields(w.shape, 21, sigma=6.0)
        g = fd.Grid(w.shape, w.spacing, w.origin)
        m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp,
                                       u_init)
        rec, uf = fd.acoustic_forward(g, so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
        torch.cuda.synchronize()
        rec, uf = rec.cpu().numpy(), uf.cpu().numpy()
        del m, sx, sw, rx, dd, ui
        og = oracle.make_grid(w.shape, w.spacing, w.origin)
        rref, uref = oracle.acoustic_forward(og, so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                             w.rec_xyz, damp=w.damp, u_init=u_init)
        assert rel_l2(uf, uref) <= TOL
        assert rel_l2(rec, rref) <= TOL
        assert max_abs_rel(uf, uref) <= TOL
        assert max_abs_rel(rec, rref) <= TOL
        del uf, uref


def test_full_size_full_run_is_linear_in_the_source():
    """512^3, so = 8, the full 1000 ms (594 steps): doubling the wavelet doubles
    every trace (FP32 scaling by 2 is exact for normal numbers; the stencil's
    numerical precursor ahead of the wavefront decays into subnormals, where
    rounding is absolute, and those last-bit differences propagate, so the
    check is to 1e-6 relative), and the field stays finite."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    w = workloads.acoustic_large(n=512, so=8)
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp)
    rec1, uf1 = fd.acoustic_forward(g, 8, w.dt, w.nt, m, sx, sw, rx, damp=dd, return_final=False)
    rec2, _ = fd.acoustic_forward(g, 8, w.dt, w.nt, m, sx, 2 * sw, rx, damp=dd,
                                  return_final=False)
    torch.cuda.synchronize()
    assert torch.isfinite(rec1).all()
    assert float(rec1.abs().max()) > 0
    scale = float(rec1.abs().max())
    assert float((rec2 - 2 * rec1).abs().max()) <= 1e-6 * 2 * scale
    assert float(torch.linalg.vector_norm(rec2 - 2 * rec1)) <= 1e-6 * float(
        torch.linalg.vector_norm(2 * rec1))
    assert w.nt == 594 and math.isclose(w.dt, 0.38 * 20.0 / 4.5)


def test_injected_values_carry_the_correctly_rounded_b():
    """From rest with unit wavelet samples, u^1 at each corner of a source is
    exactly float32(float32(w_c) * b) with b the FP32 rounding of the FP64
    value dt^2 / (m + damp dt / 2) -- for sources inside the absorbing border
    (damped nodes) and inside the interior (undamped nodes) alike."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    n, h, nbl = 48, 10.0, 8
    shape = (n, n, n)
    rng = np.random.default_rng(21)
    v = rng.uniform(1.5, 4.0, shape)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, nbl, (h, h, h), 4.0)
    dt = workloads.cfl_dt((h, h, h), 4.0)
    # one source per 3 x 3 x 3 block of cells: no two share a node
    cells = np.stack(np.meshgrid(*[np.arange(1, n - 2, 3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    cells = cells[rng.permutation(len(cells))[:300]]
    src = ((cells + rng.uniform(0.05, 0.95, cells.shape)) * h).astype(np.float32)[None]
    wav = np.ones((1, 2, src.shape[1]), np.float32)
    g = fd.Grid(shape, (h, h, h))
    mt, dd, sx, sw = to_dev(torch, m, damp, src, wav)
    e = torch.zeros((1, 0, 3), device="cuda")
    _, uf = fd.acoustic_forward(g, 4, dt, 2, mt, sx, sw, e, damp=dd)
    torch.cuda.synchronize()
    u1 = uf[0, 0].cpu().numpy()
    want = np.zeros(shape, np.float32)
    dx, dy, dz = damp[:n].astype(np.float64), damp[n:2 * n].astype(np.float64), damp[2 * n:]
    damped = 0
    for p in src[0]:
        s = p.astype(np.float64) / h
        i1 = np.floor(s).astype(int)
        fr = (s - i1).astype(np.float32)
        for c in range(8):
            ix, iy, iz = i1[0] + (c & 1), i1[1] + ((c >> 1) & 1), i1[2] + ((c >> 2) & 1)
            w = [fr[a] if (c >> a) & 1 else np.float32(1) - fr[a] for a in range(3)]
            cw = np.float32(np.float32(w[0] * w[1]) * w[2])
            d = dx[ix] + dy[iy] + float(dz[iz])
            damped += d > 0
            b = np.float32(dt * dt / (float(m[iz, iy, ix]) + 0.5 * d * dt))
            want[iz, iy, ix] = np.float32(cw * b)
    assert 0 < damped < 8 * src.shape[1]
    np.testing.assert_array_equal(u1, want)


def test_colliding_sources_are_injected_in_order_bitwise():
    """At most 16 sources per shot are injected by the stencil kernel in
    source order, so two sources on the same point give bit-identical runs,
    across tile configurations and with or without graphs."""
    require_cuda()
    from paper_1807_03032_gb300 import _native
    w, u_init = ragged_problem(8, nshots=2, nt=40)  # sources 0 and 1 coincide
    outs = []
    try:
        for cfg in range(min(3, _native.num_acoustic_configs(8))):
            _native.set_acoustic_config(8, cfg)
            outs.append(_gpu_only(w, u_init))
        _native.stats_enable(True)  # direct launches instead of graph replays
        outs.append(_gpu_only(w, u_init))
    finally:
        _native.stats_enable(False)
        _native.set_acoustic_config(8, -1)
    for rec, uf in outs[1:]:
        np.testing.assert_array_equal(uf, outs[0][1])
        np.testing.assert_array_equal(rec, outs[0][0])


def test_concurrent_calls_from_host_threads_match_sequential_runs():
    """Calls from several host threads (each on its own torch stream, device
    and host buffers, graph-replayed time loops) give the same bits as the
    same calls made one after another: the call state (private stream,
    side lanes, workspace, error text) is per call and per thread."""
    torch = require_cuda()
    import threading
    import paper_1807_03032_gb300 as fd
    cases = []
    for so, seed in ((4, 1), (8, 2), (8, 3), (4, 4)):
        w, u_init = ragged_problem(so, nshots=1, nt=40, seed=seed)
        separate_sources(w)
        cases.append((w, u_init))

    def run(w, u_init, host):
        g = fd.Grid(w.shape, w.spacing, w.origin)
        arrs = (w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp, u_init)
        if host:
            m, sx, sw, rx, dd, ui = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                                     for a in arrs]
        else:
            m, sx, sw, rx, dd, ui = to_dev(torch, *arrs)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui,
                                          stream=stream.cuda_stream)
        stream.synchronize()
        return rec.cpu().numpy(), uf.cpu().numpy()

    want = [run(w, u, host=(i % 2 == 1)) for i, (w, u) in enumerate(cases)]
    got = [None] * len(cases)
    errors = []

    def worker(i):
        try:
            for _ in range(2):
                got[i] = run(*cases[i], host=(i % 2 == 1))
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    for (rw, uw), (rg, ug) in zip(want, got):
        np.testing.assert_array_equal(rg, rw)
        np.testing.assert_array_equal(ug, uw)


@pytest.mark.parametrize("shape", [(3, 5, 7), (9, 2, 2), (2, 17, 3)])
@pytest.mark.parametrize("so", [2, 8, 16])
def test_grids_smaller_than_a_tile_and_the_stencil(shape, so):
    """Grids smaller than one tile in every axis and thinner than the stencil
    radius (most taps land on zero ghosts): FP32 storage against the oracle,
    and one binary16 step against the storage model's rounding interval."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    h = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(sum(shape) + so)
    m = workloads.slowness_squared(rng.uniform(1.5, 3.0, shape))
    damp = rng.uniform(0.0, 0.05, shape[2] + shape[1] + shape[0]).astype(np.float32)
    dt = 0.5 * workloads.cfl_dt(h, 3.0)
    u0 = rng.uniform(-1.0, 1.0, (1, 2) + shape).astype(np.float16).astype(np.float32)
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    rec = (rng.uniform(0.0, 1.0, (1, 5, 3)) * ext).astype(np.float32)
    src = (rng.uniform(0.0, 1.0, (1, 1, 3)) * ext).astype(np.float32)
    nt = 12
    wav = rng.standard_normal((1, nt, 1)).astype(np.float32)
    g = fd.Grid(shape, h)
    mt, dd, ui, sx, sw, rx = to_dev(torch, m, damp, u0, src, wav, rec)
    r, uf = fd.acoustic_forward(g, so, dt, nt, mt, sx, sw, rx, damp=dd, u_init=ui)
    torch.cuda.synchronize()
    og = oracle.make_grid(shape, h)
    ro, uo = oracle.acoustic_forward(og, so, dt, nt, m, src, wav, rec, damp=damp, u_init=u0)
    assert rel_l2(uf.cpu().numpy(), uo) <= TOL
    assert rel_l2(r.cpu().numpy(), ro) <= TOL
    # binary16 storage, one step: a rounding of a value within the FP32 error
    # bound of the exact step (the one-step check of tests/test_gpu_storage.py)
    from tests.test_gpu_storage import check_stored_step, fp32_error_bound
    e = torch.zeros((1, 0, 3), device="cuda")
    _, uh = fd.acoustic_forward(g, so, dt, 2, mt, e, torch.zeros((1, 2, 0), device="cuda"), e,
                                damp=dd, u_init=ui, storage="f16")
    torch.cuda.synchronize()
    ez = np.zeros((1, 0, 3), np.float32)
    _, ux = oracle.acoustic_forward_storage(og, so, dt, 2, m, ez, np.zeros((1, 2, 0), np.float32),
                                            ez, damp=damp, u_init=u0, storage="f16_coef")
    check_stored_step(uh.cpu().numpy()[0, 0].astype(np.float64), ux[0, 0],
                      fp32_error_bound(so, h, dt, m, u0), max_frac=0.05)
