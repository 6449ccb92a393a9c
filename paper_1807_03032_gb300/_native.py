"""ctypes binding of libfdsweep.so (the C ABI declared in include/fdsweep.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA
kernels.  There is no fallback: if the library has not been built (run
``python -m paper_1807_03032_gb300.build`` or ``__graft_entry__.build()``) or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfdsweep.so")

FD_OK = 0
STATUS_NAMES = {
    0: "FD_OK", -1: "FD_ERR_ARG", -2: "FD_ERR_CFL", -3: "FD_ERR_SO", -4: "FD_ERR_COORD",
    -5: "FD_ERR_OOM", -6: "FD_ERR_CUDA", -7: "FD_ERR_DIVERGED", -8: "FD_ERR_UNIMPL",
    -9: "FD_ERR_TIMEOUT",
}

# Every symbol include/fdsweep.h declares (checked by the ABI test).
EXPORTED = ("acoustic_forward", "tti_forward", "tti_forward_opts", "fd_last_error", "fd_version",
            "fd_stats_enable", "fd_stats_reset", "fd_stats_get", "fd_set_acoustic_config",
            "fd_num_acoustic_configs", "fd_launch_count", "acoustic_forward_noalloc",
            "acoustic_adjoint", "acoustic_gradient", "fd_engine_footprint", "fd_engine_create",
            "fd_engine_add_shot", "fd_engine_step", "fd_engine_shot_status", "fd_engine_release",
            "fd_engine_stream", "fd_engine_sync", "fd_engine_destroy", "fd_set_time_tiling",
            "fd_num_time_tiling_configs", "fd_set_tti_config", "fd_num_tti_configs",
            "acoustic_forward_opts", "fd_set_acoustic_f16_config", "fd_num_acoustic_f16_configs",
            "fd_stencil_weights", "fd_set_wait_limit_ns")


class FdGrid(ctypes.Structure):
    """Mirror of fd_grid."""

    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
                ("ox", ctypes.c_double), ("oy", ctypes.c_double), ("oz", ctypes.c_double)]


class FdTtiOptions(ctypes.Structure):
    """Mirror of fd_tti_options."""

    _fields_ = [("deriv", ctypes.c_int32), ("receiver", ctypes.c_int32),
                ("scheme", ctypes.c_int32)]


class FdAcousticOptions(ctypes.Structure):
    """Mirror of fd_acoustic_options."""

    _fields_ = [("storage", ctypes.c_int32), ("damp_layout", ctypes.c_int32)]


STORAGE = {"f32": 0, "f16": 1, "auto": 2}
DAMP_LAYOUT = {"axes": 0, "field": 1}
TTI_DERIV = {"centred": 0, "staggered": 1}
TTI_RECEIVER = {"p": 0, "mean": 1}
TTI_SCHEME = {"auto": -1, "two_pass": 0, "recompute": 1, "fused": 2}


class FdError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libfdsweep.so and declare the ABI; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(
                f"libfdsweep.so not found at {path}: build the CUDA library first "
                "(python -m paper_1807_03032_gb300.build)")
        lib = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        G = ctypes.POINTER(FdGrid)
        lib.acoustic_forward.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, P, P, P]
        lib.acoustic_forward.restype = I
        lib.acoustic_forward_opts.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, P, P,
                                              ctypes.POINTER(FdAcousticOptions), P]
        lib.acoustic_forward_opts.restype = I
        lib.fd_set_acoustic_f16_config.argtypes = [I, I]
        lib.fd_set_acoustic_f16_config.restype = I
        lib.fd_num_acoustic_f16_configs.argtypes = [I]
        lib.fd_num_acoustic_f16_configs.restype = I
        lib.acoustic_forward_noalloc.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, P, P, P]
        lib.acoustic_forward_noalloc.restype = I
        lib.acoustic_adjoint.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, P]
        lib.acoustic_adjoint.restype = I
        lib.acoustic_gradient.argtypes = [G, I, D, I, I, P, P, I, P, P, I, P, P, I, P, P]
        lib.acoustic_gradient.restype = I
        lib.tti_forward.argtypes = [G, I, D, I, I, P, P, P, P, P, P, I, P, P, I, P, P, P, P, P,
                                    P, P]
        lib.tti_forward.restype = I
        lib.tti_forward_opts.argtypes = [G, I, D, I, I, P, P, P, P, P, P, I, P, P, I, P, P, P, P,
                                         P, P, ctypes.POINTER(FdTtiOptions), P]
        lib.tti_forward_opts.restype = I
        lib.fd_last_error.argtypes = []
        lib.fd_last_error.restype = ctypes.c_char_p
        lib.fd_version.argtypes = []
        lib.fd_version.restype = ctypes.c_char_p
        lib.fd_stats_enable.argtypes = [I]
        lib.fd_stats_enable.restype = I
        lib.fd_stats_reset.argtypes = []
        lib.fd_stats_reset.restype = I
        lib.fd_stats_get.argtypes = [ctypes.c_char_p, ctypes.POINTER(D),
                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(D)]
        lib.fd_stats_get.restype = I
        lib.fd_set_tti_config.argtypes = [I, I]
        lib.fd_set_tti_config.restype = I
        lib.fd_num_tti_configs.argtypes = [I]
        lib.fd_num_tti_configs.restype = I
        lib.fd_set_time_tiling.argtypes = [I, I]
        lib.fd_set_time_tiling.restype = I
        lib.fd_num_time_tiling_configs.argtypes = [I]
        lib.fd_num_time_tiling_configs.restype = I
        lib.fd_set_acoustic_config.argtypes = [I, I]
        lib.fd_set_acoustic_config.restype = I
        lib.fd_num_acoustic_configs.argtypes = [I]
        lib.fd_num_acoustic_configs.restype = I
        VP = ctypes.POINTER(ctypes.c_void_p)
        L64 = ctypes.POINTER(ctypes.c_int64)
        IP = ctypes.POINTER(ctypes.c_int)
        lib.fd_engine_footprint.argtypes = [G, I, I, I, L64]
        lib.fd_engine_create.argtypes = [G, I, D, P, P, I, I, I, VP]
        lib.fd_engine_add_shot.argtypes = [P, I, I, P, P, I, P, P, IP]
        lib.fd_engine_step.argtypes = [P, I]
        lib.fd_engine_shot_status.argtypes = [P, I, IP, L64]
        lib.fd_engine_release.argtypes = [P, I]
        lib.fd_engine_stream.argtypes = [P, VP]
        lib.fd_engine_sync.argtypes = [P]
        lib.fd_engine_destroy.argtypes = [P]
        for name in ("fd_engine_footprint", "fd_engine_create", "fd_engine_add_shot",
                     "fd_engine_step", "fd_engine_shot_status", "fd_engine_release",
                     "fd_engine_stream", "fd_engine_sync", "fd_engine_destroy", "fd_set_time_tiling",
            "fd_num_time_tiling_configs", "fd_set_tti_config", "fd_num_tti_configs",
            "acoustic_forward_opts", "fd_set_acoustic_f16_config", "fd_num_acoustic_f16_configs",
            "fd_stencil_weights", "fd_set_wait_limit_ns"):
            getattr(lib, name).restype = I
        FP = ctypes.POINTER(ctypes.c_float)
        lib.fd_stencil_weights.argtypes = [G, I, FP, FP]
        lib.fd_set_wait_limit_ns.argtypes = [ctypes.c_int64]
        lib.fd_launch_count.argtypes = []
        lib.fd_launch_count.restype = ctypes.c_int64
        _lib = lib
        return lib


def stencil_weights(shape_zyx, spacing_xyz, so):
    """(centre, w[3][9]): the FP32 Laplacian weights of the acoustic kernels."""
    lib = load()
    c = ctypes.c_float()
    w = (ctypes.c_float * 27)()
    check(lib.fd_stencil_weights(grid_struct(shape_zyx, spacing_xyz), int(so), ctypes.byref(c),
                                 w))
    return c.value, [[w[9 * d + k] for k in range(9)] for d in range(3)]


def check(status: int):
    if status != FD_OK:
        msg = load().fd_last_error().decode(errors="replace")
        raise FdError(status, msg)


def grid_struct(shape_zyx, spacing_xyz, origin_xyz=(0.0, 0.0, 0.0)) -> FdGrid:
    nz, ny, nx = (int(v) for v in shape_zyx)
    return FdGrid(nx, ny, nz, *(float(v) for v in spacing_xyz), *(float(v) for v in origin_xyz))


def version() -> str:
    return load().fd_version().decode()


def stats_enable(on: bool = True):
    check(load().fd_stats_enable(1 if on else 0))


def stats_reset():
    check(load().fd_stats_reset())


def stats_get(family: str):
    """(total_ms, launches, points_per_launch) accumulated for a kernel family."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    pts = ctypes.c_double()
    check(load().fd_stats_get(family.encode(), ctypes.byref(ms), ctypes.byref(n),
                              ctypes.byref(pts)))
    return ms.value, n.value, pts.value


def launch_count() -> int:
    """Kernel launches enqueued by the library since it was loaded."""
    return int(load().fd_launch_count())


def set_tti_config(so: int, config: int):
    check(load().fd_set_tti_config(int(so), int(config)))


def num_tti_configs(so: int) -> int:
    return int(load().fd_num_tti_configs(int(so)))


def set_time_tiling(so: int, mode: int):
    """-1 automatic, 0 off, 1 + k on with two-step kernel configuration k."""
    check(load().fd_set_time_tiling(int(so), int(mode)))


def num_time_tiling_configs(so: int) -> int:
    return int(load().fd_num_time_tiling_configs(int(so)))


def set_acoustic_config(so: int, config: int):
    check(load().fd_set_acoustic_config(int(so), int(config)))


def num_acoustic_configs(so: int) -> int:
    return int(load().fd_num_acoustic_configs(int(so)))


def set_acoustic_f16_config(so: int, config: int):
    check(load().fd_set_acoustic_f16_config(int(so), int(config)))


def num_acoustic_f16_configs(so: int) -> int:
    return int(load().fd_num_acoustic_f16_configs(int(so)))
