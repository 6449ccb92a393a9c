"""The C-ABI library builds, loads and exports every symbol include/fdsweep.h
declares; the product path does not depend on the oracle.  No GPU needed
(no compute call is made)."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdsweep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, re.M)
    return sorted({n for n in names if n not in ("defined",)})


@pytest.fixture(scope="module")
def lib():
    from paper_1807_03032_gb300 import build, _native
    build.build()
    return _native.load()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("acoustic_forward", "tti_forward", "fd_last_error", "fd_version"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1807_03032_gb300 import _native
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) == set(_native.EXPORTED)


def test_version_and_error_string_without_gpu(lib):
    assert b"sm_103a" in lib.fd_version()
    assert isinstance(lib.fd_last_error(), bytes)


def test_config_table_queries(lib):
    from paper_1807_03032_gb300 import _native
    for so in (2, 4, 8, 12, 16):
        assert _native.num_acoustic_configs(so) >= 1
    assert _native.num_acoustic_configs(6) == 0
    with pytest.raises(_native.FdError):
        _native.set_acoustic_config(8, 99)
    _native.set_acoustic_config(8, -1)
    for so in (2, 4, 8, 12, 16):
        assert _native.num_acoustic_f16_configs(so) >= 1
    assert _native.num_acoustic_f16_configs(6) == 0
    with pytest.raises(_native.FdError):
        _native.set_acoustic_f16_config(8, 99)
    _native.set_acoustic_f16_config(8, -1)
    assert _native.stats_get("acoustic_step_h")[1] >= 0


def test_stats_api(lib):
    from paper_1807_03032_gb300 import _native
    _native.stats_reset()
    assert _native.stats_get("acoustic_step") == (0.0, 0, 0.0)
    with pytest.raises(_native.FdError):
        _native.stats_get("nonsense")


def test_product_package_does_not_import_the_oracle():
    code = ("import sys; import paper_1807_03032_gb300 as fd; "
            "assert 'oracle' not in sys.modules, 'oracle imported'; print('ok')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    pkg = os.path.join(ROOT, "paper_1807_03032_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "fd_oracle" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    from paper_1807_03032_gb300 import _native
    code = ("import paper_1807_03032_gb300._native as n\n"
            f"try:\n    n._lib=None; n.load({str(tmp_path / 'none.so')!r})\n"
            "except RuntimeError as e:\n    print('raised')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert "raised" in r.stdout, r.stdout + r.stderr
    del _native


def test_oversized_grids_are_rejected_before_any_device_work(lib):
    """A padded volume of 2^32 points or more is rejected by the host checks
    (the sparse tables index the volume in 32 bits), by every entry point
    that sizes device memory from the grid -- including the allocation-free
    call, whose scratch sizing would otherwise wrap -- with no CUDA call made
    (this runs without a GPU)."""
    import ctypes
    from paper_1807_03032_gb300 import _native
    huge = _native.grid_struct((1 << 21, 1 << 21, 1 << 21), (10.0, 10.0, 10.0),
                               (0.0, 0.0, 0.0))
    fake = ctypes.c_void_p(0x1000)  # never dereferenced: the grid check comes first
    st = lib.acoustic_forward_noalloc(huge, 4, 1.0, 4, 1, fake, None, 0, None, None, 0, None,
                                      None, None, None, None)
    assert st == {v: k for k, v in _native.STATUS_NAMES.items()}["FD_ERR_ARG"], st
    assert b"2^32" in lib.fd_last_error()
    st = lib.acoustic_forward(huge, 4, 1.0, 4, 1, fake, None, 0, None, None, 0, None, None,
                              None, None, None)
    assert st == {v: k for k, v in _native.STATUS_NAMES.items()}["FD_ERR_ARG"], st
    out = ctypes.c_void_p()
    st = lib.fd_engine_create(huge, 8, 1.0, fake, None, 1, 1, 1, ctypes.byref(out))
    assert st == {v: k for k, v in _native.STATUS_NAMES.items()}["FD_ERR_ARG"], st
    nbytes = ctypes.c_int64()
    st = lib.fd_engine_footprint(huge, 1, 1, 1, ctypes.byref(nbytes))
    assert st == {v: k for k, v in _native.STATUS_NAMES.items()}["FD_ERR_ARG"], st
    # a non-finite origin is rejected the same way
    bad = _native.grid_struct((8, 8, 8), (10.0, 10.0, 10.0), (float("nan"), 0.0, 0.0))
    st = lib.acoustic_forward_noalloc(bad, 4, 1.0, 4, 1, fake, None, 0, None, None, 0, None,
                                      None, None, None, None)
    assert st == {v: k for k, v in _native.STATUS_NAMES.items()}["FD_ERR_ARG"], st


@pytest.mark.parametrize("so", [2, 4, 8, 12, 16])
@pytest.mark.parametrize("spacing", [(20.0, 20.0, 20.0), (9.0, 11.0, 10.0), (5.0, 5.0, 12.5)])
def test_device_laplacian_weights_sum_to_zero_exactly(so, spacing):
    """The FP32 weights the acoustic kernels use: the Laplacian of a constant
    is exactly zero (checked in exact rational arithmetic), as it is for the
    closed-form weights (w_0 = -2 sum w_k, Listing fd-1 for so = 2); every
    weight differs from the FP32 rounding of its exact value by at most one
    ulp of the centre weight (the size of the residual that was moved), and
    each axis keeps the second moment sum_k 2 k^2 w_k h^2 = 2 of a second
    derivative to 1e-6 (a phase velocity error below 5e-7).  With
    independently rounded weights the residual is a spurious mass term whose
    phase error grows linearly in time (1.1e-4 relative L2 after the 1000 ms
    acoustic workload at so = 12)."""
    from fractions import Fraction
    import numpy as np
    from paper_1807_03032_gb300 import _native
    from tests.fd_exact import second_derivative_weights
    centre, w = _native.stencil_weights((8, 8, 8), spacing, so)
    R = so // 2
    total = Fraction(centre) + 2 * sum(Fraction(w[d][k]) for d in range(3) for k in range(1, 9))
    assert total == 0
    exact = second_derivative_weights(R)  # Fractions, index 0..R
    want_c = float(sum(exact[0] / Fraction(h) ** 2 for h in spacing))
    ulp_c = float(np.spacing(np.float32(abs(want_c))))
    assert abs(centre - float(np.float32(want_c))) <= ulp_c
    for d in range(3):
        assert w[d][0] == 0.0
        for k in range(1, 9):
            want = float(exact[k] / Fraction(spacing[d]) ** 2) if k <= R else 0.0
            got = w[d][k]
            if k > R:
                assert got == 0.0
                continue
            assert abs(got - float(np.float32(want))) <= ulp_c, (d, k, got, want)
        moment = sum(2 * k * k * Fraction(w[d][k]) for k in range(1, R + 1)) * Fraction(
            spacing[d]) ** 2
        assert abs(float(moment) - 2.0) <= 1e-6 * 2.0
