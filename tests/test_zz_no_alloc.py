"""hope_total_mass_noalloc: the mass diagnostic for callers that cannot allocate device
memory (for example a host framework whose device-memory budget is fixed after start-up,
or a loop that cannot afford the synchronisation an allocation may cause).  It is called through the C ABI and must
agree with hope_total_mass, the context-based entry point, on two calls in a row (the
second call reuses the static scratch left by the first).

This file is collected last on purpose, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MASS_RTOL = 1e-14  # the tolerance of the other mass-diagnostic tests


@pytest.fixture(scope="module")
def hp():
    import paper_2411_19185_gb300 as hp
    hp.load()
    return hp


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_mass_matches_context_mass_twice(hp, precision):
    lib = hp._lib.load()
    prec = hp.HOPE_FP64 if precision == "fp64" else hp.HOPE_FP32
    N = 20
    s = hp.Sphere(N, 5, precision=prec)
    q = s.rossby_haurwitz()
    ref = s.mass(q)  # hope_total_mass (context scratch)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        rc = lib.hope_total_mass_noalloc(ctypes.c_void_p(q.data_ptr()), prec, N,
                                         ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                         stream)
        assert rc == 0, lib.hope_last_error_message()
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= MASS_RTOL * abs(ref), (got, ref)
        out.fill_(float("nan"))
    s.close()


def test_noalloc_mass_rejects_sizes_beyond_the_scratch(hp):
    lib = hp._lib.load()
    q = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = 1183  # one more than HOPE_NOALLOC_MASS_MAX_N: rejected before any launch
    rc = lib.hope_total_mass_noalloc(ctypes.c_void_p(q.data_ptr()), hp.HOPE_FP64, big,
                                     ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                     None)
    assert rc == -1
    assert b"static scratch" in lib.hope_last_error_message()


def _noalloc(lib, q, prec, N, out):
    rc = lib.hope_total_mass_noalloc(ctypes.c_void_p(q.data_ptr()), prec, N,
                                     ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.hope_last_error_message()
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_mass_at_the_largest_size_matches_an_exact_host_sum(hp):
    """The whole static scratch in use: N = HOPE_NOALLOC_MASS_MAX_N (4096 partial sums of
    2048 elements, FP32 state of about 100 MB) on a seeded positive state, against the
    correctly rounded sum of the same FP32 values on the host (math.fsum) times dx^2;
    then a small sphere (which reuses only the first slots left by the large call) and the
    large one again."""
    import math
    import numpy as np
    lib = hp._lib.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for N in (1182, 7, 1182):
        rng = np.random.default_rng(N)
        q = (1.0 + rng.random((3, 6, N, N))).astype(np.float32)
        exact = math.fsum(q[0].astype(np.float64).ravel().tolist()) * (math.pi / (2 * N)) ** 2
        got = _noalloc(lib, torch.from_numpy(q).cuda(), hp.HOPE_FP32, N, out)
        assert abs(got - exact) <= 1e-12 * exact, (N, got, exact)  # one partial missing: 2.4e-4
