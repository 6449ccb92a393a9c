"""Binary16 storage of the acoustic path (acoustic_forward_opts, storage
"f16") against the oracle's storage model.

Both sides round every stored value to binary16; the device decides each
rounding on its FP32 result and the oracle on its FP64 result rounded to FP32,
so the two stored values agree except where the exact value lies within the
FP32 evaluation error of a rounding midpoint (or where the update cancels so
far that the binary16 spacing falls below that error).  One step from a rough
random state checks at every point that the device's value is a rounding of
a value within the FP32 error bound of the exact one.  Over many steps the differing decisions propagate; the run is
then checked against the size of the storage error itself (the distance of
the storage model from the unrounded model).
"""
import numpy as np
import pytest

import oracle
import workloads
from tests.gpu_util import rel_l2, require_cuda, to_dev

pytestmark = pytest.mark.gpu


def as_f16(x):
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def one_step_case(so, shape=(29, 27, 70), seed=4, h=(10.0, 9.0, 11.0)):
    """Rough random medium and state (every value a binary16 value), damping,
    no sources or receivers; nx = 70 gives a partial second 64-wide tile and
    a row padded from 70 to 72 halves."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(1.5, 3.5, shape)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 5, h, 3.5)
    dt = 0.9 * workloads.cfl_dt(h, 3.5)
    u = as_f16(rng.uniform(-1.0, 1.0, (1, 2) + tuple(shape))).astype(np.float32)
    return shape, h, m, damp, dt, u


def gpu_run(torch, shape, h, so, dt, nt, m, damp, u_init=None, src=None, wav=None, rec=None,
            storage="f16", nshots=1):
    import paper_1807_03032_gb300 as fd
    src = np.zeros((nshots, 0, 3), np.float32) if src is None else src
    wav = np.zeros((nshots, nt, 0), np.float32) if wav is None else wav
    rec = np.zeros((nshots, 0, 3), np.float32) if rec is None else rec
    g = fd.Grid(shape, h)
    mt, dd, ui, sx, sw, rx = to_dev(torch, m, damp, u_init, src, wav, rec)
    r, uf = fd.acoustic_forward(g, so, dt, nt, mt, sx, sw, rx, damp=dd, u_init=ui,
                                storage=storage)
    torch.cuda.synchronize()
    return r.cpu().numpy().astype(np.float64), uf.cpu().numpy().astype(np.float64)


def fp32_error_bound(so, h, dt, m, u):
    """Absolute bound on the FP32 evaluation error of one update: a few
    rounding units (2^-24) per operation of the (6R + 8)-term chain, times
    the largest magnitude that enters it, |u| + |u-| + b sum |w_k| |u| / h^2."""
    r = so // 2
    w, _ = oracle.fd_weights(r)
    wsum = abs(w[0]) + 2 * sum(abs(x) for x in w[1:])
    bmax = dt * dt / float(m.min())
    umax = float(np.abs(u).max())
    scale = 2 * umax + bmax * wsum * sum(1.0 / x ** 2 for x in h) * umax
    return 4 * (6 * r + 8) * 2.0 ** -24 * scale


def check_stored_step(got, exact, bound, max_frac=0.02):
    """got: device result; exact: the oracle's unrounded FP64 value with the
    same binary16 inputs.  The device stores the binary16 rounding of an FP32
    value within `bound` of the exact one, and rounding is monotone, so every
    stored value must lie between the roundings of exact - bound and exact +
    bound.  Away from cancellation that allows only the adjacent value, and
    only near a rounding midpoint; where the update cancels to far below its
    inputs (binary16 spacing under the FP32 error) it allows a few spacings.
    Few points may round differently from the oracle at all."""
    want = as_f16(exact.astype(np.float32))
    frac = float((got != want).mean())
    assert frac <= max_frac, frac
    lo, hi = as_f16(exact - bound), as_f16(exact + bound)
    bad = (got < lo) | (got > hi)
    assert not bad.any(), (int(bad.sum()), got[bad][:5], exact[bad][:5])
    return frac


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
def test_one_step_rounding_decisions(so):
    torch = require_cuda()
    shape, h, m, damp, dt, u = one_step_case(so)
    _, uf = gpu_run(torch, shape, h, so, dt, 2, m, damp, u_init=u)
    np.testing.assert_array_equal(uf[0, 1], u[0, 0])  # u^0 passes through unchanged
    og = oracle.make_grid(shape, h)
    e = np.zeros((1, 0, 3), np.float32)
    _, ux = oracle.acoustic_forward_storage(og, so, dt, 2, m, e, np.zeros((1, 2, 0), np.float32),
                                            e, damp=damp, u_init=u, storage="f16_coef")
    frac = check_stored_step(uf[0, 0], ux[0, 0], fp32_error_bound(so, h, dt, m, u))
    print(f"so {so}: {frac:.2e} of the points rounded the other way")


def test_every_tile_configuration_agrees_bitwise():
    torch = require_cuda()
    from paper_1807_03032_gb300 import _native
    for so in (2, 4, 8, 12, 16):
        shape, h, m, damp, dt, u = one_step_case(so, seed=9)
        outs = []
        try:
            for cfg in range(_native.num_acoustic_f16_configs(so)):
                _native.set_acoustic_f16_config(so, cfg)
                outs.append(gpu_run(torch, shape, h, so, dt, 5, m, damp, u_init=u)[1])
        finally:
            _native.set_acoustic_f16_config(so, -1)
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])


def test_no_step_returns_rounded_initial_state_and_traces():
    torch = require_cuda()
    shape, h, m, damp, dt, u = one_step_case(8)
    rng = np.random.default_rng(1)
    u = (rng.standard_normal(u.shape) * 3.0).astype(np.float32)  # not binary16 values
    ext = np.array([(shape[2] - 1) * h[0], (shape[1] - 1) * h[1], (shape[0] - 1) * h[2]])
    rec = (rng.uniform(0, 1, (1, 40, 3)) * ext).astype(np.float32)
    r, uf = gpu_run(torch, shape, h, 8, dt, 1, m, damp, u_init=u, rec=rec)
    np.testing.assert_array_equal(uf[0], as_f16(u[0]))
    og = oracle.make_grid(shape, h)
    e = np.zeros((1, 0, 3), np.float32)
    ro, _ = oracle.acoustic_forward_storage(og, 8, dt, 1, m, e, np.zeros((1, 1, 0), np.float32),
                                            rec, damp=damp, u_init=u, storage="f16")
    assert rel_l2(r, ro) <= 1e-6


def run_case(so, nt=80, shape=(40, 36, 70), h=10.0, seed=2):
    shape = tuple(shape)
    v = workloads.smooth_random(shape, seed, 3.0, 1.5, 3.0)
    m = workloads.slowness_squared(v)
    damp = workloads.damping_profile(shape, 6, (h, h, h), 3.0)
    dt = workloads.cfl_dt((h, h, h), 3.0)
    ext = np.array([(shape[2] - 1) * h, (shape[1] - 1) * h, (shape[0] - 1) * h])
    src = (np.array([[[0.41, 0.52, 0.45]]]) * ext).astype(np.float32)
    xs = np.linspace(0.1, 0.9, 48) * ext[0]
    rec = np.stack([xs, np.full(48, 0.33 * ext[1]), np.full(48, 0.3 * ext[2])], -1)[None]
    wav = workloads.ricker(nt, dt, f0=0.03)[None, :, None].astype(np.float32)
    return shape, (h, h, h), m, damp, dt, src, wav, rec.astype(np.float32)


@pytest.mark.parametrize("so", [4, 8, 16])
def test_run_is_as_accurate_as_the_storage_model(so):
    """80 steps with a source, receivers and damping.  A rounding decision
    that went the other way (a few 1e-4 of the points per step, by one
    binary16 spacing) makes the two states differ; from then on the
    roundings at the affected points are decided on different values, so the
    device run and the storage model become two realisations of the same
    rounding noise, spreading with the wave.  Hence: the device run is as far
    from the unrounded model as the storage model is (within 1.5x), and the
    two differ by at most the difference of two such realisations (2x, above
    the sqrt(2) of independent noise)."""
    torch = require_cuda()
    shape, h, m, damp, dt, src, wav, rec = run_case(so)
    nt = wav.shape[1]
    rg, ug = gpu_run(torch, shape, h, so, dt, nt, m, damp, src=src, wav=wav, rec=rec)
    og = oracle.make_grid(shape, h)
    rm, um = oracle.acoustic_forward_storage(og, so, dt, nt, m, src, wav, rec, damp=damp,
                                             storage="f16")
    rx, ux = oracle.acoustic_forward_storage(og, so, dt, nt, m, src, wav, rec, damp=damp,
                                             storage="exact")
    for got, model, exact in ((rg, rm, rx), (ug, um, ux)):
        e_model = rel_l2(model, exact)
        assert e_model > 2.0 ** -14  # the rounding is visible
        print(f"so {so}: model {e_model:.3e}, device vs model {rel_l2(got, model):.3e}, "
              f"device vs unrounded {rel_l2(got, exact):.3e}")
        assert rel_l2(got, exact) <= 1.5 * e_model, (rel_l2(got, exact), e_model)
        assert rel_l2(got, model) <= 2.0 * e_model, (rel_l2(got, model), e_model)


def test_shots_are_independent_and_runs_repeat_bitwise():
    torch = require_cuda()
    shape, h, m, damp, dt, src, wav, rec = run_case(8, nt=30)
    src2 = np.concatenate([src, src * np.float32(0.8)], 0)
    wav2 = np.concatenate([wav, -0.5 * wav], 0)
    rec2 = np.concatenate([rec, rec[:, ::-1]], 0)
    r2, u2 = gpu_run(torch, shape, h, 8, dt, 30, m, damp, src=src2, wav=wav2, rec=rec2,
                     nshots=2)
    for s in range(2):
        r1, u1 = gpu_run(torch, shape, h, 8, dt, 30, m, damp, src=src2[s:s + 1],
                         wav=wav2[s:s + 1], rec=rec2[s:s + 1])
        np.testing.assert_array_equal(r2[s], r1[0])
        np.testing.assert_array_equal(u2[s], u1[0])


def test_f32_storage_through_the_options_entry_is_acoustic_forward():
    torch = require_cuda()
    shape, h, m, damp, dt, src, wav, rec = run_case(8, nt=20)
    a = gpu_run(torch, shape, h, 8, dt, 20, m, damp, src=src, wav=wav, rec=rec, storage="f32")
    import paper_1807_03032_gb300 as fd
    g = fd.Grid(shape, h)
    mt, dd, sx, sw, rx = to_dev(torch, m, damp, src, wav, rec)
    r, uf = fd.acoustic_forward(g, 8, dt, 20, mt, sx, sw, rx, damp=dd)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(a[0], r.cpu().numpy())
    np.testing.assert_array_equal(a[1], uf.cpu().numpy())


def test_overflow_is_reported_as_diverged():
    torch = require_cuda()
    from paper_1807_03032_gb300 import _native
    shape, h, m, damp, dt, u = one_step_case(4)
    u = np.empty_like(u)
    u[0, 0] = 60000.0
    u[0, 1] = -60000.0   # u + (u - u-) is far above the largest binary16 value
    with pytest.raises(_native.FdError) as ei:
        gpu_run(torch, shape, h, 4, dt, 3, m, damp, u_init=u)
    assert ei.value.name == "FD_ERR_DIVERGED"


def test_bad_storage_and_statistics_family():
    torch = require_cuda()
    import ctypes
    import paper_1807_03032_gb300 as fd
    from paper_1807_03032_gb300 import _native
    shape, h, m, damp, dt, src, wav, rec = run_case(4, nt=6)
    g = fd.Grid(shape, h)
    mt, dd, sx, sw, rx = to_dev(torch, m, damp, src, wav, rec)
    out = torch.empty((1, 6, rec.shape[1]), device="cuda")
    opts = _native.FdAcousticOptions(7)
    st = _native.load().acoustic_forward_opts(
        g.struct(), 4, float(dt), 6, 1, mt.data_ptr(), dd.data_ptr(), 1, sx.data_ptr(),
        sw.data_ptr(), rec.shape[1], rx.data_ptr(), out.data_ptr(), None, None,
        ctypes.byref(opts), None)
    assert _native.STATUS_NAMES[st] == "FD_ERR_ARG"
    _native.stats_reset()
    _native.stats_enable(True)
    try:
        gpu_run(torch, shape, h, 4, dt, 6, m, damp, src=src, wav=wav, rec=rec)
    finally:
        _native.stats_enable(False)
    ms, n, pts = _native.stats_get("acoustic_step_h")
    assert n == 5 and pts == float(np.prod(shape)) and ms > 0


def test_full_size_one_step_at_512():
    """The 512^3 benchmark grid in the launch configuration the benchmark
    times (so = 8, h = 20 m, smooth 1.5-4.5 km/s model, 40-point border):
    one step from a random binary16 state, every point checked."""
    torch = require_cuda()
    w = workloads.acoustic_large(n=512, so=8, nt=2)
    rng = np.random.default_rng(12)
    u = as_f16(rng.uniform(-1.0, 1.0, (1, 2) + tuple(w.shape))).astype(np.float32)
    _, uf = gpu_run(torch, w.shape, w.spacing, 8, w.dt, 2, w.m, w.damp, u_init=u)
    og = oracle.make_grid(w.shape, w.spacing, w.origin)
    e = np.zeros((1, 0, 3), np.float32)
    _, ux = oracle.acoustic_forward_storage(og, 8, w.dt, 2, w.m, e,
                                            np.zeros((1, 2, 0), np.float32), e, damp=w.damp,
                                            u_init=u, storage="f16_coef")
    np.testing.assert_array_equal(uf[0, 1], u[0, 0])
    check_stored_step(uf[0, 0], ux[0, 0], fp32_error_bound(8, w.spacing, w.dt, w.m, u))


def test_host_buffers_give_the_same_bits():
    """Host (pinned and pageable) inputs and outputs go through the same
    device path: traces and final fields identical to the device-buffer run."""
    torch = require_cuda()
    import paper_1807_03032_gb300 as fd
    shape, h, m, damp, dt, src, wav, rec = run_case(8, nt=40)
    u0 = as_f16(workloads.random_wavefields(shape, 5, nshots=1, amplitude=0.01)).astype(np.float32)
    rd, ud = gpu_run(torch, shape, h, 8, dt, 40, m, damp, u_init=u0, src=src, wav=wav, rec=rec)
    g = fd.Grid(shape, h)
    for pinned in (False, True):
        arrs = [torch.from_numpy(np.ascontiguousarray(a)) for a in (m, damp, src, wav, rec, u0)]
        if pinned:
            arrs = [a.pin_memory() for a in arrs]
        mh, dh, sh, wh, rh, uh = arrs
        r, uf = fd.acoustic_forward(g, 8, dt, 40, mh, sh, wh, rh, damp=dh, u_init=uh,
                                    storage="f16")
        torch.cuda.synchronize()
        assert not r.is_cuda and not uf.is_cuda
        np.testing.assert_array_equal(r.numpy(), rd)
        np.testing.assert_array_equal(uf.numpy(), ud)


@pytest.mark.parametrize("so", [4, 8, 12, 16])
def test_automatic_storage_picks_the_faster_kernel_per_space_order(so):
    """FD_STORAGE_AUTO: binary16 storage for so <= 8, FP32 for so 12 and 16,
    bit for bit the run of the storage it chose."""
    torch = require_cuda()
    shape, h, m, damp, dt, src, wav, rec = run_case(so, nt=16)
    auto = gpu_run(torch, shape, h, so, dt, 16, m, damp, src=src, wav=wav, rec=rec,
                   storage="auto")
    want = gpu_run(torch, shape, h, so, dt, 16, m, damp, src=src, wav=wav, rec=rec,
                   storage="f16" if so <= 8 else "f32")
    np.testing.assert_array_equal(auto[0], want[0])
    np.testing.assert_array_equal(auto[1], want[1])
