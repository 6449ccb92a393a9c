"""GB300-native (sm_103a) finite-difference wave-propagation sweep.

The time-stepped 3-D stencil operators that Devito (arXiv:1807.03032) generates
and benchmarks -- isotropic acoustic and TTI forward modelling with sparse
source injection and receiver interpolation -- as hand-written CUDA kernels
behind a small C ABI (``include/fdsweep.h``).  This module is the thin Python
binding: it marshals PyTorch tensors (device or host) or NumPy arrays into the
C calls and allocates outputs; all arithmetic runs in the CUDA kernels.

Conventions: arrays are C order [z][y][x]; coordinates are (x, y, z) in m;
time in ms; velocity in km/s; m = 1/v^2.
"""
from __future__ import annotations

import ctypes

from dataclasses import dataclass

import numpy as np

from . import _native
from ._native import FdError, stats_enable, stats_get, stats_reset, version  # noqa: F401

__all__ = ["Grid", "acoustic_forward", "acoustic_adjoint", "acoustic_gradient", "tti_forward",
           "FdError", "version", "stats_enable", "stats_get", "stats_reset"]


@dataclass(frozen=True)
class Grid:
    """The paper's Grid(shape, extent, origin): shape (nz, ny, nx) including the
    absorbing border, spacing (hx, hy, hz) and origin (ox, oy, oz) in metres."""

    shape: tuple
    spacing: tuple
    origin: tuple = (0.0, 0.0, 0.0)

    def struct(self):
        return _native.grid_struct(self.shape, self.spacing, self.origin)


def _torch():
    import torch
    return torch


def _is_tensor(x):
    try:
        torch = _torch()
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


def _ptr(x, name):
    if x is None:
        return None
    if _is_tensor(x):
        torch = _torch()
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 tensor")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags.c_contiguous:
            raise TypeError(f"{name} must be a C-contiguous float32 array")
        return x.ctypes.data
    raise TypeError(f"{name}: expected a torch.Tensor or numpy.ndarray, got {type(x)!r}")


def _empty_like_kind(ref, shape):
    if _is_tensor(ref):
        torch = _torch()
        return torch.empty(shape, dtype=torch.float32, device=ref.device)
    return np.empty(shape, dtype=np.float32)


def _stream_for(*arrays, stream=None):
    if stream is not None:
        return int(stream)
    for a in arrays:
        if _is_tensor(a) and a.is_cuda:
            torch = _torch()
            return torch.cuda.current_stream(a.device).cuda_stream
    return 0


def _as_grid(grid):
    return grid if isinstance(grid, Grid) else Grid(*grid)


def acoustic_forward(grid, so, dt, nt, m, src_xyz, src_wav, rec_xyz, damp=None, u_init=None,
                     rec_out=None, u_final=None, return_final=True, stream=None, storage="f32",
                     damp_layout="axes"):
    """Isotropic acoustic forward model (C ABI ``acoustic_forward``).

    m [nz][ny][nx]; damp [nx+ny+nz] per-axis profiles (damp_layout "axes")
    or a 3-D field [nz][ny][nx] ("field": C ABI ``acoustic_forward_opts``
    with FD_DAMP_FIELD), or None;
    src_xyz [nshots][nsrc][3]; src_wav [nshots][nt][nsrc]; rec_xyz [nshots][nrec][3];
    u_init [nshots][2][nz][ny][nx] (u^0, u^-1) or None.
    storage: "f32", "f16" (wavefields and b held in IEEE binary16 on the
    device, FP32 arithmetic; C ABI ``acoustic_forward_opts``) or "auto"
    (binary16 for so <= 8, where it is the faster storage on GB300, FP32
    beyond).
    Returns (rec [nshots][nt][nrec], u_final [nshots][2][nz][ny][nx] or None).
    Outputs are allocated like ``m`` (same device / host) unless given.
    """
    g = _as_grid(grid)
    nshots, nsrc = int(src_xyz.shape[0]), int(src_xyz.shape[1])
    nrec = int(rec_xyz.shape[1])
    if rec_xyz.shape[0] != nshots or src_wav.shape[0] != nshots:
        raise ValueError("src_xyz, src_wav and rec_xyz must share the shot dimension")
    if tuple(src_wav.shape[1:]) != (nt, nsrc):
        raise ValueError("src_wav must be [nshots][nt][nsrc]")
    if rec_out is None:
        rec_out = _empty_like_kind(m, (nshots, nt, nrec))
    if u_final is None and return_final:
        u_final = _empty_like_kind(m, (nshots, 2) + tuple(g.shape))
    lib = _native.load()
    args = (g.struct(), int(so), float(dt), int(nt), nshots, _ptr(m, "m"), _ptr(damp, "damp"),
            nsrc, _ptr(src_xyz, "src_xyz"), _ptr(src_wav, "src_wav"), nrec,
            _ptr(rec_xyz, "rec_xyz"), _ptr(rec_out, "rec_out"), _ptr(u_init, "u_init"),
            _ptr(u_final, "u_final"))
    stream_ptr = _stream_for(m, rec_out, stream=stream)
    if storage == "f32" and damp_layout == "axes":
        st = lib.acoustic_forward(*args, stream_ptr)
    else:
        opts = _native.FdAcousticOptions(_native.STORAGE[storage],
                                         _native.DAMP_LAYOUT[damp_layout])
        st = lib.acoustic_forward_opts(*args, ctypes.byref(opts), stream_ptr)
    _native.check(st)
    return rec_out, u_final


def tti_forward(grid, so, dt, nt, m, eps, delta, theta, phi, src_xyz, src_wav, rec_xyz,
                damp=None, p_init=None, r_init=None, rec_out=None, p_final=None, r_final=None,
                return_final=True, stream=None, deriv="centred", receiver="p",
                scheme="auto"):
    """TTI forward model (C ABI ``tti_forward``, or ``tti_forward_opts`` for the
    alternative readings).  deriv: "centred" | "staggered"; receiver: "p" |
    "mean" ((p + r)/2); scheme: "auto" | "fused" (temporaries in shared
    memory, so <= 8) | "two_pass" (temporaries in device memory) |
    "recompute" (no temporaries).  Returns (rec, p_final, r_final)."""
    g = _as_grid(grid)
    nshots, nsrc = int(src_xyz.shape[0]), int(src_xyz.shape[1])
    nrec = int(rec_xyz.shape[1])
    if tuple(src_wav.shape[1:]) != (nt, nsrc):
        raise ValueError("src_wav must be [nshots][nt][nsrc]")
    if rec_out is None:
        rec_out = _empty_like_kind(m, (nshots, nt, nrec))
    if return_final:
        if p_final is None:
            p_final = _empty_like_kind(m, (nshots, 2) + tuple(g.shape))
        if r_final is None:
            r_final = _empty_like_kind(m, (nshots, 2) + tuple(g.shape))
    lib = _native.load()
    args = (g.struct(), int(so), float(dt), int(nt), nshots, _ptr(m, "m"), _ptr(damp, "damp"),
            _ptr(eps, "eps"), _ptr(delta, "delta"), _ptr(theta, "theta"), _ptr(phi, "phi"),
            nsrc, _ptr(src_xyz, "src_xyz"), _ptr(src_wav, "src_wav"), nrec,
            _ptr(rec_xyz, "rec_xyz"), _ptr(rec_out, "rec_out"), _ptr(p_init, "p_init"),
            _ptr(r_init, "r_init"), _ptr(p_final, "p_final"), _ptr(r_final, "r_final"))
    stream_ptr = _stream_for(m, rec_out, stream=stream)
    if (deriv, receiver, scheme) == ("centred", "p", "auto"):
        st = lib.tti_forward(*args, stream_ptr)
    else:
        opts = _native.FdTtiOptions(_native.TTI_DERIV[deriv], _native.TTI_RECEIVER[receiver],
                                    _native.TTI_SCHEME[scheme])
        st = lib.tti_forward_opts(*args, ctypes.byref(opts), stream_ptr)
    _native.check(st)
    return rec_out, p_final, r_final


def acoustic_adjoint(grid, so, dt, nt, m, src_xyz, rec_xyz, rec_resid, damp=None, src_grad=None,
                     stream=None):
    """Adjoint of acoustic_forward's source-to-receiver map (C ABI
    ``acoustic_adjoint``): residual traces [nshots][nt][nrec] -> adjoint source
    wavelets [nshots][nt][nsrc] (allocated like ``m`` unless given)."""
    g = _as_grid(grid)
    nshots, nsrc = int(src_xyz.shape[0]), int(src_xyz.shape[1])
    nrec = int(rec_xyz.shape[1])
    if tuple(rec_resid.shape) != (nshots, nt, nrec):
        raise ValueError("rec_resid must be [nshots][nt][nrec]")
    if src_grad is None:
        src_grad = _empty_like_kind(m, (nshots, nt, nsrc))
    st = _native.load().acoustic_adjoint(
        g.struct(), int(so), float(dt), int(nt), nshots, _ptr(m, "m"), _ptr(damp, "damp"), nsrc,
        _ptr(src_xyz, "src_xyz"), _ptr(src_grad, "src_grad"), nrec, _ptr(rec_xyz, "rec_xyz"),
        _ptr(rec_resid, "rec_resid"), _stream_for(m, src_grad, stream=stream))
    _native.check(st)
    return src_grad


def acoustic_gradient(grid, so, dt, nt, m, src_xyz, src_wav, rec_xyz, rec_resid, damp=None,
                      checkpoint_every=0, grad=None, stream=None):
    """Gradient with respect to m of <rec_resid, d(m)> (C ABI
    ``acoustic_gradient``), checkpointing the forward wavefield every
    ``checkpoint_every`` steps (0: sqrt(nt-1)).  Returns [nz][ny][nx]."""
    g = _as_grid(grid)
    nshots, nsrc = int(src_xyz.shape[0]), int(src_xyz.shape[1])
    nrec = int(rec_xyz.shape[1])
    if tuple(rec_resid.shape) != (nshots, nt, nrec):
        raise ValueError("rec_resid must be [nshots][nt][nrec]")
    if tuple(src_wav.shape) != (nshots, nt, nsrc):
        raise ValueError("src_wav must be [nshots][nt][nsrc]")
    if grad is None:
        grad = _empty_like_kind(m, tuple(g.shape))
    st = _native.load().acoustic_gradient(
        g.struct(), int(so), float(dt), int(nt), nshots, _ptr(m, "m"), _ptr(damp, "damp"), nsrc,
        _ptr(src_xyz, "src_xyz"), _ptr(src_wav, "src_wav"), nrec, _ptr(rec_xyz, "rec_xyz"),
        _ptr(rec_resid, "rec_resid"), int(checkpoint_every), _ptr(grad, "grad"),
        _stream_for(m, grad, stream=stream))
    _native.check(st)
    return grad
