"""Shared helpers of the GPU parity tests."""
import numpy as np
import pytest

TOL = 1e-4  # relative L2, wavefields and traces, GPU FP32 vs oracle FP64


def rel_l2(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor, 1e-300))


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_03032_gb300 import build, _native
    build.build()
    _native.load()
    return torch


def to_dev(torch, *arrays):
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
            for a in arrays]


def max_abs_rel(a, b):
    """max |a - b| / max |b|: a single wrong point in a large field moves the
    relative L2 distance by little, but shows here."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))
