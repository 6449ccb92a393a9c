"""Time tiling (two leapfrog steps per launch, fd_set_time_tiling): results
bit-identical to single steps, parity with the oracle, fallbacks."""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import TOL, rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def problem(so, nt, nshots=2, nsrc=3, seed=11, shape=(100, 37, 70)):
    """Ragged box: nx = 70 (two x tiles, the second partial), ny = 37 (three y
    tiles), nz = 100 (split into z chunks); anisotropic spacing, shifted
    origin, damping, random initial state, sources on distinct nodes."""
    h = (9.0, 11.0, 10.0)
    o = (-100.0, 250.0, 30.0)
    rng = np.random.default_rng(seed)
    v = 1.5 + 2.0 * workloads.smooth_random(shape, seed, 3.0, 0.0, 1.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 6, h, 3.5)
    dt = 0.9 * workloads.cfl_dt(h, 3.5)
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    src = o + rng.uniform(0.02, 0.98, (nshots, nsrc, 3)) * ext
    src[:, 0, :2] = o[:2]          # a source on the x = y = origin edge
    rec = o + rng.uniform(0.0, 1.0, (nshots, 23, 3)) * ext
    rec[:, 0] = o + ext
    wav = rng.standard_normal((nshots, nt, nsrc))
    u_init = 1e-2 * workloads.random_wavefields(shape, seed, nshots=nshots, sigma=2.0)
    w = workloads.Workload("tt", shape, h, o, so, dt, nt, m, damp, src.astype(np.float32),
                           wav.astype(np.float32), rec.astype(np.float32))
    return w, u_init


def run_gpu(w, u_init, mode, stats=False):
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    g = fd.Grid(w.shape, w.spacing, w.origin)
    m, sx, sw, rx, dd, ui = to_dev(torch, w.m, w.src_xyz, w.src_wav, w.rec_xyz, w.damp, u_init)
    _native.set_time_tiling(w.so, mode)
    if stats:
        _native.stats_reset()
        _native.stats_enable(True)
    try:
        rec, uf = fd.acoustic_forward(g, w.so, w.dt, w.nt, m, sx, sw, rx, damp=dd, u_init=ui)
        torch.cuda.synchronize()
    finally:
        _native.set_time_tiling(w.so, -1)
        if stats:
            _native.stats_enable(False)
    return rec.cpu().numpy(), uf.cpu().numpy()


def configs(so):
    require_cuda()
    from paper_1807_03032_gb300 import _native
    return range(_native.num_time_tiling_configs(so))


@pytest.mark.parametrize("so", [4, 8])
@pytest.mark.parametrize("nt", [31, 70])
def test_two_step_kernel_bit_identical_to_single_steps(so, nt):
    """Every configuration of the two-step kernel, with graphs (default) and
    with direct launches (statistics mode), an even and an odd number of
    steps (nt = 70 replays graphs and ends with a single step): traces and
    final fields equal those of single steps bit for bit."""
    w, u_init = problem(so, nt)
    ref = run_gpu(w, u_init, 0)
    assert np.linalg.norm(ref[0]) > 0
    for k in configs(so):
        for stats in (False, True):
            got = run_gpu(w, u_init, 1 + k, stats=stats)
            np.testing.assert_array_equal(got[1], ref[1])
            np.testing.assert_array_equal(got[0], ref[0])


def test_two_step_kernel_used_and_counted():
    from paper_1807_03032_gb300 import _native
    w, u_init = problem(4, 32, nshots=1)  # 31 steps: 15 pairs and one single step
    run_gpu(w, u_init, 1, stats=True)
    ms, n, pts = _native.stats_get("acoustic_step2")
    assert n == 15 and ms > 0 and pts == float(np.prod(w.shape))
    ms1, n1, _ = _native.stats_get("acoustic_step")
    assert n1 == 1


@pytest.mark.parametrize("so", [4, 8])
def test_time_tiled_parity_with_oracle(so):
    w, u_init = problem(so, 41, shape=(40, 37, 70))
    rec, uf = run_gpu(w, u_init, 1)
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    rref, uref = oracle.acoustic_forward(og, w.so, w.dt, w.nt, w.m, w.src_xyz, w.src_wav,
                                         w.rec_xyz, damp=w.damp, u_init=u_init)
    assert rel_l2(uf, uref) <= TOL
    assert rel_l2(rec, rref) <= TOL


def test_many_sources_fall_back_to_single_steps():
    """More sources per shot than the two-step kernel injects: the forced mode
    falls back to single steps (same result, no two-step launch)."""
    from paper_1807_03032_gb300 import _native
    w, u_init = problem(4, 12, nshots=1, nsrc=20)
    ref = run_gpu(w, u_init, 0)
    got = run_gpu(w, u_init, 1, stats=True)
    np.testing.assert_array_equal(got[1], ref[1])
    assert _native.stats_get("acoustic_step2")[1] == 0


def test_bad_mode_rejected():
    require_cuda()
    from paper_1807_03032_gb300 import _native
    with pytest.raises(_native.FdError):
        _native.set_time_tiling(4, 99)
    with pytest.raises(_native.FdError):
        _native.set_time_tiling(5, 0)
    _native.set_time_tiling(4, -1)
