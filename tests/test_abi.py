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
    assert lib.hope_init_grid(32, 7, _lib.HOPE_WENO1D, ctypes.byref(p), ctypes.byref(h)) == -6  # comparator: order 5
    p.precision = 9
    assert lib.hope_init_grid(32, 5, 0, ctypes.byref(p), ctypes.byref(h)) == -1
    assert not h.value
    assert lib.hope_strerror(-1) == b"invalid argument"
    assert b"invalid" in lib.hope_last_error_message()
    assert lib.hope_tendency(None, None, None, None) == -1
    assert lib.hope_step(None, None, 1.0, 1, None) == -1
    assert lib.hope_set_topography(None, None) == -1
    assert b"null context" in lib.hope_last_error_message()
    assert lib.hope_initial_state(None, 11, None, 0, None, 0, None, None) == -1


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


@pytest.mark.parametrize("N,k,prec", [(8, 3, 0), (10, 5, 0), (9, 7, 0), (10, 5, 1), (12, 11, 0), (9, 9, 1)])
def test_ghost_operator_storage_selfcheck_on_host(lib, N, k, prec):
    """The ghost operator built on the host (no GPU) is stored as rotated copies of panel-0
    representatives: every composed row equals its representative's image to 1e-12, and
    the stored form, applied as the ghost kernel applies it (columns with symmetry codes,
    representative weights; FP64 head and FP32 tail), equals the full operator on a seeded
    state to 1e-13 (FP64 contexts: the tail's FP32 weights) or exactly (FP32 contexts)."""
    s, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    rc = lib.hope_ghost_selfcheck(N, k, prec, ctypes.byref(s), ctypes.byref(a), ctypes.byref(b))
    assert rc == 0
    assert s.value == 1
    assert a.value < 1e-12
    assert b.value < (1e-13 if prec == 0 else 1e-15)


def test_ghost_selfcheck_rejects_invalid_arguments(lib):
    s, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    for args in [(0, 5, 0), (10, 4, 0), (10, 13, 0), (10, 5, 2)]:
        assert lib.hope_ghost_selfcheck(*args, ctypes.byref(s), ctypes.byref(a), ctypes.byref(b)) == -1  # EINVAL


def test_ghost_storage_falls_back_when_rows_are_not_images(lib):
    """A stencil wider than the panel (N = 7, k = 9) amplifies round-off in the composed
    rows beyond the 1e-12 acceptance, so every row keeps its own weights (identity codes)
    and the stored form is the full operator exactly."""
    s, a, b = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    assert lib.hope_ghost_selfcheck(7, 9, 0, ctypes.byref(s), ctypes.byref(a), ctypes.byref(b)) == 0
    assert s.value == 0 and a.value > 1e-12 and b.value == 0.0
