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
