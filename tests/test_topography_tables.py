"""The library's bottom-surface tables (built on the host in FP64, no GPU) against the
oracle: the surface's values at the edge points, and psi_B's cell average (eq. 2.14) as
the tables' affine map of the depth stencil, on section 5.2's mountain and flow with 1%
depth noise.  The GPU kernels that apply the tables are checked by the -m gpu tests."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from synth import noise_field, perturb_h


@pytest.fixture(scope="module")
def lib():
    from paper_2411_19185_gb300 import build as B
    B.build()
    from paper_2411_19185_gb300 import _lib
    return _lib.load()


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@pytest.mark.parametrize("N,k,tol", [(13, 3, 1e-12), (17, 5, 1e-12), (12, 11, 1e-10)])
def test_tables_match_oracle(lib, N, k, tol):
    """sep: 1e-13 of the surface's scale.  psi_B: relative L2 per component `tol` (measured
    5e-14 for k <= 5, 1.4e-12 for k = 11): the oracle takes the gradient of phi_t from the
    reconstruction of depth + surface, the tables split it into the depth stencil's
    weights and the surface's constant, which partly cancel over the mountain (the
    balanced free surface is flatter than the bottom), and the 11-point derivative
    weights' alternating signs amplify the rounding of both routes."""
    o = O.Oracle(N, k)
    o.set_mountain()
    q = o.geostrophic(u0=20.0, phi0=5960.0 * O.GRAVITY)
    q = np.ascontiguousarray(perturb_h(q, noise_field((6, N, N), 2)))
    sbar = np.ascontiguousarray(o.topography())
    me, H, kk = (k + 1) // 2, (k - 1) // 2, k * k
    pn = 6 * N * N
    sep, w, b = np.empty(4 * me * pn), np.empty(2 * kk * pn), np.empty(2 * pn)
    assert lib.hope_topography_tables(N, k, O.RADIUS, _ptr(sbar), _ptr(sep), _ptr(w), _ptr(b)) == 0
    sep, w, b = sep.reshape(4, me, 6, N, N), w.reshape(2, kk, 6, N, N), b.reshape(2, 6, N, N)
    # edge values of the surface against the oracle's reconstruction of it
    z = np.zeros((3, 6, N, N))
    z[0] = sbar
    exs, _ = o.fill_ghosts(z)
    spts = o.reconstruct_all(exs)[0]  # [6][N][N][n_poc]
    got = np.stack([sep[s_][r] for s_ in range(4) for r in range(me)], axis=-1)
    assert np.max(np.abs(got - spts[..., :4 * me])) < 1e-13 * np.max(np.abs(spts))
    # psi_B = b + sum_c w[c] * stencil_c of the depth (the oracle's ghost fill of q)
    ext = o.fill_ghosts(q)[0][0]  # [6][ne][ne]
    psib = b.copy()
    for bb in range(k):
        for a in range(k):
            psib += w[:, bb * k + a] * ext[None, :, bb:bb + N, a:a + N]
    ref = o.topo_psib(q)
    for v in range(2):
        rel = np.linalg.norm(psib[v] - ref[v]) / np.linalg.norm(ref[v])
        assert rel < tol, (v, rel)


def test_oracle_psib_is_linear_in_the_surface_at_fixed_phi_t():
    """psi_B = sqrtG phi_s G^ij d_j phi_t: with the same free surface phi_t (the initial
    conditions read their phi as phi_t) a surface twice as high gives twice the source,
    and no surface gives none."""
    N, k = 10, 5
    p = []
    for hs0 in (300.0, 600.0):
        o = O.Oracle(N, k)
        o.set_mountain(hs0=hs0)
        p.append(o.topo_psib(o.geostrophic(u0=20.0, phi0=5960.0 * O.GRAVITY)))
    assert np.linalg.norm(p[1] - 2 * p[0]) < 1e-12 * np.linalg.norm(p[0])
    flat = O.Oracle(N, k)
    assert not np.any(flat.topo_psib(flat.geostrophic(u0=20.0, phi0=5960.0 * O.GRAVITY)))


def test_tables_reject_bad_arguments(lib):
    s = np.zeros(6 * 8 * 8)
    assert lib.hope_topography_tables(2, 3, O.RADIUS, _ptr(s), None, None, None) == -1
    assert lib.hope_topography_tables(8, 4, O.RADIUS, _ptr(s), None, None, None) == -1
    assert lib.hope_topography_tables(8, 3, 0.0, _ptr(s), None, None, None) == -1
    assert lib.hope_topography_tables(8, 3, O.RADIUS, None, None, None, None) == -1
