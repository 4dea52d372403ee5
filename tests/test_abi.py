"""C-ABI checks that need no GPU: the library loads, exports every function that
include/hope.h declares, and rejects invalid arguments with HOPE_EINVAL before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_19185_gb300 import build as B
    B.build()
    from paper_2411_19185_gb300 import _lib
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "hope.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hope_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_all_exported(lib):
    from paper_2411_19185_gb300 import _lib
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTED)


def test_invalid_arguments_rejected_without_device(lib):
    from paper_2411_19185_gb300 import _lib
    h = ctypes.c_void_p()
    p = _lib.default_params()
    assert lib.hope_init_grid(32, 4, 0, ctypes.byref(p), ctypes.byref(h)) == _lib.HOPE_OK - 1  # even order
    assert lib.hope_init_grid(2, 5, 0, ctypes.byref(p), ctypes.byref(h)) == -1  # N < order
    assert lib.hope_init_grid(32, 5, 7, ctypes.byref(p), ctypes.byref(h)) == -1  # bad scheme
    p.precision = 9
    assert lib.hope_init_grid(32, 5, 0, ctypes.byref(p), ctypes.byref(h)) == -1
    assert not h.value
    assert lib.hope_strerror(-1) == b"invalid argument"
    assert b"invalid" in lib.hope_last_error_message()
    assert lib.hope_tendency(None, None, None, None) == -1
    assert lib.hope_step(None, None, 1.0, 1, None) == -1


def test_default_params(lib):
    from paper_2411_19185_gb300 import _lib
    p = _lib.default_params()
    assert p.radius == 6.37122e6 and p.gravity == 9.80616 and p.omega == 7.292e-5
    assert p.ghost_iters == 10 and p.precision == 0 and p.rk == 0


def test_product_path_has_no_oracle_import():
    """The product package never imports, loads or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2411_19185_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dp, f)).read()
                assert "oracle" not in txt.lower(), os.path.join(dp, f)
