"""FP64 CPU oracle for the FD wave-propagation sweep (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA path and never imports it.

The arithmetic lives in ``fd_oracle.c`` (plain loops in FP64, compiled with gcc
and ``-ffp-contract=off`` so that no fused multiply-add changes a rounding);
this module only builds that file and marshals NumPy arrays into it.  Every
function cites the passage of the paper it follows in the C source.

Parity: every function exported here is pinned by a ``-m "not gpu"`` test
(``tests/test_oracle_*.py``) against a closed form, an exact rational
computation, an invariant or a special case; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Grid(ctypes.Structure):
    """Grid descriptor: shape incl. the damping border, spacing, origin."""

    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("hx", ctypes.c_double),
        ("hy", ctypes.c_double),
        ("hz", ctypes.c_double),
        ("ox", ctypes.c_double),
        ("oy", ctypes.c_double),
        ("oz", ctypes.c_double),
    ]


def make_grid(shape_zyx, spacing_xyz, origin_xyz=(0.0, 0.0, 0.0)) -> Grid:
    nz, ny, nx = (int(v) for v in shape_zyx)
    hx, hy, hz = (float(v) for v in spacing_xyz)
    ox, oy, oz = (float(v) for v in origin_xyz)
    return Grid(nx, ny, nz, hx, hy, hz, ox, oy, oz)


def build(force: bool = False) -> str:
    """Compile fd_oracle.c into _build/liboracle.so (for this machine)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            G = ctypes.POINTER(Grid)
            lib.ora_fd_weights.argtypes = [I, P, P]
            lib.ora_fd_weights.restype = None
            lib.ora_laplacian.argtypes = [G, I, I, P, P]
            lib.ora_first_derivative.argtypes = [G, I, I, I, P, P]
            lib.ora_first_derivative_kind.argtypes = [G, I, I, I, I, P, P]
            lib.ora_staggered_weights.argtypes = [I, P]
            lib.ora_staggered_weights.restype = None
            lib.ora_acoustic_step.argtypes = [G, I, I, D, P, P, P, P, P]
            lib.ora_interpolate.argtypes = [G, I, P, P, P]
            lib.ora_inject.argtypes = [G, I, P, P, P, P]
            lib.ora_acoustic_forward.argtypes = [G, I, I, D, I, I, P, P, I, P, P, I, P, P, P, P]
            lib.ora_acoustic_forward_field.argtypes = [G, I, I, D, I, I, P, P, I, P, P, I, P, P,
                                                       P, P]
            lib.ora_tti_operators.argtypes = [G, I, I, P, P, P, P, P]
            lib.ora_tti_operators_kind.argtypes = [G, I, I, I, P, P, P, P, P]
            lib.ora_tti_forward.argtypes = [G, I, I, D, I, I, P, P, P, P, P, P,
                                            I, P, P, I, P, P, P, P, P, P]
            lib.ora_tti_forward_opts.argtypes = [G, I, I, I, I, D, I, I, P, P, P, P, P, P,
                                                 I, P, P, I, P, P, P, P, P, P]
            lib.ora_tti_forward_storage.argtypes = [G, I, I, D, I, I, P, P, P, P, P, P,
                                                    I, P, P, I, P, P, P, P, P, P, I]
            lib.ora_acoustic_adjoint.argtypes = [G, I, I, D, I, I, P, P, I, P, P, I, P, P]
            lib.ora_round_binary16.argtypes = [D]
            lib.ora_round_binary16.restype = D
            lib.ora_acoustic_forward_storage.argtypes = [G, I, I, D, I, I, P, P, I, P, P, I, P,
                                                         P, P, P, I]
            lib.ora_acoustic_gradient.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, P]
            for name in ("ora_acoustic_adjoint", "ora_acoustic_gradient",
                         "ora_laplacian", "ora_first_derivative", "ora_acoustic_step",
                         "ora_interpolate", "ora_inject", "ora_acoustic_forward",
                         "ora_acoustic_forward_field",
                         "ora_tti_operators", "ora_tti_forward", "ora_first_derivative_kind",
                         "ora_tti_operators_kind", "ora_tti_forward_opts", "ora_tti_forward_storage",
                         "ora_acoustic_forward_storage"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def fd_weights(r: int):
    """(w, c): second- and first-derivative central weights for radius r."""
    lib = _load()
    w = np.zeros(r + 1)
    c = np.zeros(r + 1)
    lib.ora_fd_weights(int(r), _ptr(w), _ptr(c))
    return w, c


def laplacian(grid: Grid, so: int, u, periodic: bool = False):
    u = _f64(u)
    out = np.empty_like(u)
    _check(_load().ora_laplacian(ctypes.byref(grid), so, int(periodic), _ptr(u), _ptr(out)),
           "laplacian")
    return out


def staggered_weights(r: int):
    """Staggered first-derivative weights [0, a_1..a_r] for radius r."""
    a = np.zeros(r + 1)
    _load().ora_staggered_weights(int(r), _ptr(a))
    return a


_KINDS = {"central": 0, "forward": 1, "backward": -1}


def first_derivative(grid: Grid, so: int, axis: int, f, periodic: bool = False,
                     kind: str = "central"):
    """axis 0 = x, 1 = y, 2 = z (arrays are [z][y][x]).  kind: "central",
    "forward" (staggered D+, value at i + 1/2) or "backward" (D-, at i - 1/2)."""
    f = _f64(f)
    out = np.empty_like(f)
    lib = _load()
    if kind == "central":
        st = lib.ora_first_derivative(ctypes.byref(grid), so, int(periodic), axis, _ptr(f),
                                      _ptr(out))
    else:
        st = lib.ora_first_derivative_kind(ctypes.byref(grid), so, int(periodic), axis,
                                           _KINDS[kind], _ptr(f), _ptr(out))
    _check(st, "first_derivative")
    return out


def acoustic_step(grid: Grid, so: int, dt: float, m, u, uprev, damp=None,
                  periodic: bool = False):
    m, u, uprev = _f64(m), _f64(u), _f64(uprev)
    damp = None if damp is None else _f64(damp)
    out = np.empty_like(u)
    _check(_load().ora_acoustic_step(ctypes.byref(grid), so, int(periodic), float(dt), _ptr(m),
                                     _ptr(damp), _ptr(u), _ptr(uprev), _ptr(out)),
           "acoustic_step")
    return out


def interpolate(grid: Grid, xyz, u):
    xyz = _f32(xyz)
    u = _f64(u)
    npt = xyz.shape[0]
    out = np.empty(npt)
    _check(_load().ora_interpolate(ctypes.byref(grid), npt, _ptr(xyz), _ptr(u), _ptr(out)),
           "interpolate")
    return out


def inject(grid: Grid, xyz, q, scale, u):
    """Return u + injection of q (per point) with per-node `scale`."""
    xyz = _f32(xyz)
    q = _f64(q)
    scale = _f64(scale)
    out = _f64(u).copy()
    _check(_load().ora_inject(ctypes.byref(grid), xyz.shape[0], _ptr(xyz), _ptr(q), _ptr(scale),
                              _ptr(out)), "inject")
    return out


def acoustic_forward(grid: Grid, so: int, dt: float, nt: int, m, src_xyz, src_wav, rec_xyz,
                     damp=None, u_init=None, periodic: bool = False, damp_layout: str = "axes"):
    """Full acoustic forward run.

    src_xyz [nshots][nsrc][3], src_wav [nshots][nt][nsrc], rec_xyz [nshots][nrec][3],
    u_init [nshots][2][nz][ny][nx] or None; damp per-axis profiles [nx+ny+nz]
    (damp_layout "axes") or a 3-D field [nz][ny][nx] ("field").  Returns
    (rec [nshots][nt][nrec], u_final [nshots][2][nz][ny][nx]) in FP64.
    """
    m = _f32(m)
    damp = _f32(damp)
    src_xyz, src_wav, rec_xyz = _f32(src_xyz), _f32(src_wav), _f32(rec_xyz)
    u_init = _f32(u_init)
    nshots, nsrc = src_xyz.shape[0], src_xyz.shape[1]
    nrec = rec_xyz.shape[1]
    rec = np.zeros((nshots, nt, nrec))
    ufin = np.zeros((nshots, 2) + m.shape)
    fn = {"axes": _load().ora_acoustic_forward,
          "field": _load().ora_acoustic_forward_field}[damp_layout]
    st = fn(ctypes.byref(grid), so, int(periodic), float(dt), int(nt), nshots, _ptr(m),
            _ptr(damp), nsrc, _ptr(src_xyz), _ptr(src_wav), nrec, _ptr(rec_xyz), _ptr(rec),
            _ptr(u_init), _ptr(ufin))
    _check(st, "acoustic_forward")
    return rec, ufin


_STORAGE = {"exact": 0, "f16": 1, "f16_coef": 2}


def round_binary16(x):
    """Nearest IEEE binary16 value of each element (ties to even), FP64 out."""
    x = np.asarray(x, dtype=np.float64)
    f = _load().ora_round_binary16
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float64])(x) if x.size else x.copy()


def acoustic_forward_storage(grid: Grid, so: int, dt: float, nt: int, m, src_xyz, src_wav,
                             rec_xyz, damp=None, u_init=None, storage: str = "f16",
                             periodic: bool = False):
    """Acoustic forward model with reduced-precision storage.

    storage "f16": the wavefield levels and the coefficient b = dt^2/(m +
    damp dt/2) are stored in IEEE binary16 (values the device computes in FP32
    are rounded to FP32, then to binary16); "f16_coef": only b is stored in
    binary16, the wavefields stay exact (one step of it, rounded, is one step
    of "f16"); "exact": no rounding (the same model as acoustic_forward,
    update written in the b form).  Shapes and return values as
    acoustic_forward.
    """
    m = _f32(m)
    damp = _f32(damp)
    src_xyz, src_wav, rec_xyz = _f32(src_xyz), _f32(src_wav), _f32(rec_xyz)
    u_init = _f32(u_init)
    nshots, nsrc = src_xyz.shape[0], src_xyz.shape[1]
    nrec = rec_xyz.shape[1]
    rec = np.zeros((nshots, nt, nrec))
    ufin = np.zeros((nshots, 2) + m.shape)
    st = _load().ora_acoustic_forward_storage(
        ctypes.byref(grid), so, int(periodic), float(dt), int(nt), nshots, _ptr(m), _ptr(damp),
        nsrc, _ptr(src_xyz), _ptr(src_wav), nrec, _ptr(rec_xyz), _ptr(rec), _ptr(u_init),
        _ptr(ufin), _STORAGE[storage])
    _check(st, "acoustic_forward_storage")
    return rec, ufin


_DERIVS = {"centred": 0, "staggered": 1}
_RECEIVERS = {"p": 0, "mean": 1}


def tti_operators(grid: Grid, so: int, theta, phi, q, periodic: bool = False,
                  deriv: str = "centred"):
    """(Hz q, L q) for the rotated TTI operators (deriv "centred" or "staggered")."""
    theta, phi, q = _f64(theta), _f64(phi), _f64(q)
    hz = np.empty_like(q)
    lq = np.empty_like(q)
    lib = _load()
    if deriv == "centred":
        st = lib.ora_tti_operators(ctypes.byref(grid), so, int(periodic), _ptr(theta),
                                   _ptr(phi), _ptr(q), _ptr(hz), _ptr(lq))
    else:
        st = lib.ora_tti_operators_kind(ctypes.byref(grid), so, int(periodic), _DERIVS[deriv],
                                        _ptr(theta), _ptr(phi), _ptr(q), _ptr(hz), _ptr(lq))
    _check(st, "tti_operators")
    return hz, lq


def tti_forward(grid: Grid, so: int, dt: float, nt: int, m, eps, delta, theta, phi, src_xyz,
                src_wav, rec_xyz, damp=None, p_init=None, r_init=None, periodic: bool = False,
                deriv: str = "centred", receiver: str = "p", storage: str = "exact"):
    """Full TTI forward run.  Returns (rec, p_final, r_final) in FP64.
    deriv: "centred" or "staggered"; receiver: "p" or "mean" ((p + r)/2).
    storage: "exact" (the FP64 model) or "f32" (a yardstick for FP32 storage:
    a and s rounded to FP32, p and r rounded to FP32 after every step;
    central derivatives and receivers on p only)."""
    m, eps, delta, theta, phi = (_f32(a) for a in (m, eps, delta, theta, phi))
    damp = _f32(damp)
    src_xyz, src_wav, rec_xyz = _f32(src_xyz), _f32(src_wav), _f32(rec_xyz)
    p_init, r_init = _f32(p_init), _f32(r_init)
    nshots, nsrc = src_xyz.shape[0], src_xyz.shape[1]
    nrec = rec_xyz.shape[1]
    rec = np.zeros((nshots, nt, nrec))
    pfin = np.zeros((nshots, 2) + m.shape)
    rfin = np.zeros((nshots, 2) + m.shape)
    lib = _load()
    if storage != "exact":
        if (deriv, receiver, storage) != ("centred", "p", "f32"):
            raise ValueError("storage='f32' takes central derivatives and receivers on p")
        st = lib.ora_tti_forward_storage(
            ctypes.byref(grid), so, int(periodic), float(dt), int(nt), nshots, _ptr(m), _ptr(damp),
            _ptr(eps), _ptr(delta), _ptr(theta), _ptr(phi), nsrc, _ptr(src_xyz), _ptr(src_wav),
            nrec, _ptr(rec_xyz), _ptr(rec), _ptr(p_init), _ptr(r_init), _ptr(pfin), _ptr(rfin), 1)
    elif deriv == "centred" and receiver == "p":
        st = lib.ora_tti_forward(ctypes.byref(grid), so, int(periodic), float(dt), int(nt),
                                 nshots, _ptr(m), _ptr(damp), _ptr(eps), _ptr(delta), _ptr(theta),
                                 _ptr(phi), nsrc, _ptr(src_xyz), _ptr(src_wav), nrec,
                                 _ptr(rec_xyz), _ptr(rec), _ptr(p_init), _ptr(r_init),
                                 _ptr(pfin), _ptr(rfin))
    else:
        st = lib.ora_tti_forward_opts(ctypes.byref(grid), so, int(periodic), _DERIVS[deriv],
                                      _RECEIVERS[receiver], float(dt), int(nt), nshots, _ptr(m),
                                      _ptr(damp), _ptr(eps), _ptr(delta), _ptr(theta), _ptr(phi),
                                      nsrc, _ptr(src_xyz), _ptr(src_wav), nrec, _ptr(rec_xyz),
                                      _ptr(rec), _ptr(p_init), _ptr(r_init), _ptr(pfin),
                                      _ptr(rfin))
    _check(st, "tti_forward")
    return rec, pfin, rfin


def acoustic_adjoint(grid: Grid, so: int, dt: float, nt: int, m, src_xyz, rec_xyz, rec_resid,
                     damp=None, periodic: bool = False):
    """Adjoint of the source-to-receiver map of `acoustic_forward` (zero initial
    state): receiver residuals [nshots][nt][nrec] -> source-wavelet gradient
    [nshots][nt][nsrc] (FP64)."""
    m = _f32(m)
    damp = _f32(damp)
    src_xyz, rec_xyz = _f32(src_xyz), _f32(rec_xyz)
    rr = _f64(rec_resid)
    nshots, nsrc = src_xyz.shape[0], src_xyz.shape[1]
    nrec = rec_xyz.shape[1]
    out = np.zeros((nshots, nt, nsrc))
    st = _load().ora_acoustic_adjoint(ctypes.byref(grid), so, int(periodic), float(dt), int(nt),
                                      nshots, _ptr(m), _ptr(damp), nsrc, _ptr(src_xyz), _ptr(out),
                                      nrec, _ptr(rec_xyz), _ptr(rr))
    _check(st, "acoustic_adjoint")
    return out


def acoustic_gradient(grid: Grid, so: int, dt: float, nt: int, m, src_xyz, src_wav, rec_xyz,
                      rec_resid, damp=None):
    """Gradient with respect to m of <rec_resid, d(m)> summed over shots
    ([nz][ny][nx], FP64); with rec_resid = d(m) - d_obs it is the gradient of
    J(m) = 1/2 ||d(m) - d_obs||^2."""
    m = _f32(m)
    damp = _f32(damp)
    src_xyz, src_wav, rec_xyz = _f32(src_xyz), _f32(src_wav), _f32(rec_xyz)
    rr = _f64(rec_resid)
    nshots, nsrc = src_xyz.shape[0], src_xyz.shape[1]
    nrec = rec_xyz.shape[1]
    grad = np.zeros(m.shape)
    st = _load().ora_acoustic_gradient(ctypes.byref(grid), so, float(dt), int(nt), nshots,
                                       _ptr(m), _ptr(damp), nsrc, _ptr(src_xyz), _ptr(src_wav),
                                       nrec, _ptr(rec_xyz), _ptr(rr), _ptr(grad))
    _check(st, "acoustic_gradient")
    return grad
