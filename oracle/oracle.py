"""TEST INFRASTRUCTURE ONLY: ctypes binding of the plain C oracle (hope_oracle.c).

The oracle is a plain, slow FP64 CPU implementation of the HOPE cubed-sphere
shallow-water spatial operator (arXiv 2411.19185, sections 2-3) used to check the
CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may use it.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hope_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TPP, WENO, WENO1D = 0, 1, 2
SSPRK3, WSRK3 = 0, 1
IC_GEOSTROPHIC, IC_ROSSBY, IC_DAMBREAK, IC_BUMPS, IC_GALEWSKY = 2, 6, 7, 8, 11
# section 5.4: umax, theta0, theta1, theta2, alpha, beta, hhat; phi0 = 0: mean depth 10 km
GALEWSKY = (80.0, np.pi / 7, 5 * np.pi / 14, np.pi / 4, 1.0 / 3, 1.0 / 15, 120.0)
TOPO_MOUNTAIN, TOPO_ZONAL, TOPO_HILL = 1, 2, 3

RADIUS = 6.37122e6
GRAVITY = 9.80616
OMEGA = 7.292e-5


def build_oracle(force=False):
    """Compile the C oracle with gcc (OpenMP) into oracle/liboracle.so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "hope_oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        L.orc_new.restype = vp
        L.orc_new.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_free.argtypes = [vp]
        L.orc_set_coriolis_tilt.argtypes = [vp, ctypes.c_double]
        L.orc_npoc.argtypes = [vp]
        L.orc_halo.argtypes = [vp]
        L.orc_tendency.argtypes = [vp, P, P]
        L.orc_tendency_cells.argtypes = [vp, P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), P]
        L.orc_step.argtypes = [vp, P, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.orc_mass.restype = ctypes.c_double
        L.orc_mass.argtypes = [vp, P]
        L.orc_fill_ghosts.argtypes = [vp, P, P, P]
        L.orc_reconstruct_all.argtypes = [vp, P, P]
        L.orc_ic.argtypes = [vp, ctypes.c_int, P, ctypes.c_int, P, P]
        L.orc_cell_sqrtg.argtypes = [vp, P]
        L.orc_ic_point.argtypes = [vp, ctypes.c_int, P, ctypes.c_double, ctypes.c_double, P]
        L.orc_norms.argtypes = [vp, P, P, P]
        L.orc_gauss.argtypes = [ctypes.c_int, P, P]
        L.orc_weights_1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, P]
        L.orc_tpp_weights_2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        L.orc_tpp_weights_2d_literal.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        L.orc_weno_gamma.restype = ctypes.c_int
        L.orc_weno_gamma.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
        L.orc_weno_beta.restype = ctypes.c_double
        L.orc_weno_beta.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.orc_weno1d_gamma.restype = ctypes.c_int
        L.orc_weno1d_gamma.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
        L.orc_weno1d_point.restype = ctypes.c_double
        L.orc_weno1d_point.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_double]
        L.orc_weno_point.restype = ctypes.c_double
        L.orc_weno_point.argtypes = [vp, P, ctypes.c_int]
        L.orc_metric.argtypes = [ctypes.c_double, ctypes.c_double, P]
        L.orc_jacobian.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        L.orc_xyz.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, P]
        L.orc_locate.restype = ctypes.c_int
        L.orc_locate.argtypes = [P, P]
        L.orc_lmars.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P, P]
        L.orc_sources.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P]
        L.orc_lmars_topo.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P,
                                     ctypes.c_double, ctypes.c_double, P]
        L.orc_set_topography.argtypes = [vp, P]
        L.orc_set_topography_case.argtypes = [vp, ctypes.c_int, P]
        L.orc_get_topography.argtypes = [vp, P]
        L.orc_topography_point.restype = ctypes.c_double
        L.orc_topography_point.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_topo_psib.argtypes = [vp, P, P]
        L.orc_set_topography_form.argtypes = [vp, ctypes.c_int]
        L.orc_tpp_dweights_2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, P]
        L.orc_sqrtg_grad.argtypes = [ctypes.c_double, ctypes.c_double, P]
        Pi = ctypes.POINTER(ctypes.c_int)
        L.orc_ghost_count.restype = ctypes.c_int
        L.orc_ghost_count.argtypes = [vp]
        L.orc_ghost_tables.argtypes = [vp, Pi, Pi, Pi, Pi, P, P, P, P, P]
        L.orc_edge_tables.argtypes = [vp, Pi, Pi, Pi, Pi, P, P]
        L.orc_coriolis.restype = ctypes.c_double
        L.orc_coriolis.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Oracle:
    """One grid of the oracle: N cells per panel edge, stencil width k (odd), scheme TPP/WENO."""

    def __init__(self, N, k, scheme=TPP, radius=RADIUS, gravity=GRAVITY, omega=OMEGA,
                 weno_eps=1e-40, ghost_iters=10, coriolis_tilt=0.0):
        self.N, self.k, self.scheme = N, k, scheme
        self.radius, self.gravity, self.omega = radius, gravity, omega
        self._h = lib().orc_new(N, k, scheme, radius, gravity, omega, weno_eps, ghost_iters)
        if not self._h:
            raise ValueError("oracle: invalid grid N=%d k=%d" % (N, k))
        lib().orc_set_coriolis_tilt(self._h, float(coriolis_tilt))
        self.coriolis_tilt = float(coriolis_tilt)
        self.H = (k - 1) // 2
        self.me = (k + 1) // 2
        self.npoc = lib().orc_npoc(self._h)
        self.dx = np.pi / (2 * N)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    @property
    def shape(self):
        return (3, 6, self.N, self.N)

    def tendency(self, q):
        q = _f64(q)
        out = np.empty(self.shape)
        lib().orc_tendency(self._h, _p(q), _p(out))
        return out

    def tendency_cells(self, q, cells):
        """L(q) at the flat cell indices p*N*N + j*N + i only, shape (3, len(cells)): the
        tendency's computation with the reconstruction restricted to what those cells need."""
        q = _f64(q)
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        assert cells.ndim == 1 and cells.size and cells.min() >= 0 and cells.max() < 6 * self.N ** 2
        out = np.empty((3, cells.size))
        lib().orc_tendency_cells(self._h, _p(q), int(cells.size),
                                 cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(out))
        return out

    def step(self, q, dt, nsteps=1, rk=SSPRK3):
        q = _f64(q).copy()
        lib().orc_step(self._h, _p(q), float(dt), int(nsteps), int(rk))
        return q

    def mass(self, q):
        return lib().orc_mass(self._h, _p(_f64(q)))

    def fill_ghosts(self, q):
        q = _f64(q)
        ne = self.N + 2 * self.H
        ext = np.empty((3, 6, ne, ne))
        res = np.empty(3)
        lib().orc_fill_ghosts(self._h, _p(q), _p(ext), _p(res))
        return ext, res

    def reconstruct_all(self, ext):
        ext = _f64(ext)
        pts = np.empty((3, 6, self.N, self.N, self.npoc))
        lib().orc_reconstruct_all(self._h, _p(ext), _p(pts))
        return pts

    def ic(self, case, params, extra=None):
        params = _f64(list(np.ravel(params)) + [0.0] * max(0, 8 - np.size(params)))
        extra = _f64(np.zeros(1) if extra is None else np.ravel(extra))
        n_extra = extra.size if case == IC_BUMPS else 0
        out = np.empty(self.shape)
        lib().orc_ic(self._h, int(case), _p(params), int(n_extra), _p(extra), _p(out))
        return out

    def geostrophic(self, alpha=0.0, u0=None, phi0=2.94e4):
        if u0 is None:
            u0 = 2 * np.pi * self.radius / (12 * 86400.0)
        return self.ic(IC_GEOSTROPHIC, [alpha, u0, phi0])

    def rossby_haurwitz(self, w=7.848e-6, K=7.848e-6, R=4.0, h0=8000.0):
        return self.ic(IC_ROSSBY, [w, K, R, h0])

    def dam_break(self, lon=0.0, lat=0.0, radius=np.deg2rad(20.0), h_in=10.0, h_out=1.0):
        return self.ic(IC_DAMBREAK, [lon, lat, radius, h_in, h_out])

    def galewsky(self, perturbed=True, phi0=0.0):
        """The perturbed jet of section 5.4 (eqs. 5.16-5.18); perturbed=False drops phi'."""
        P = list(GALEWSKY)
        if not perturbed:
            P[6] = 0.0
        return self.ic(IC_GALEWSKY, P + [phi0])

    def ic_point(self, case, params, lam, th):
        P = _f64(list(params) + [0.0] * (8 - len(params)))
        out = np.empty(3)
        lib().orc_ic_point(self._h, int(case), _p(P), float(lam), float(th), _p(out))
        return out

    def bumps(self, centres, alpha=0.0, amp=50.0, radius=np.deg2rad(5.0), u0=None, phi0=2.94e4):
        if u0 is None:
            u0 = 2 * np.pi * self.radius / (12 * 86400.0)
        c = _f64(centres).reshape(-1, 2)
        return self.ic(IC_BUMPS, [alpha, u0, phi0, amp, radius], c.ravel())

    def cell_sqrtg(self):
        out = np.empty((6, self.N, self.N))
        lib().orc_cell_sqrtg(self._h, _p(out))
        return out

    def norms(self, q, qref):
        out = np.empty(3)
        lib().orc_norms(self._h, _p(_f64(q)), _p(_f64(qref)), _p(out))
        return out

    def weno_point(self, stencil, pt):
        return lib().orc_weno_point(self._h, _p(_f64(stencil).ravel()), int(pt))

    def lmars(self, direction, X, Y, qL, qR):
        F = np.empty(3)
        lib().orc_lmars(self._h, int(direction), float(X), float(Y), _p(_f64(qL)), _p(_f64(qR)), _p(F))
        return F

    def sources(self, panel, X, Y, q):
        S = np.empty(3)
        lib().orc_sources(self._h, int(panel), float(X), float(Y), _p(_f64(q)), _p(S))
        return S

    def ghost_tables(self):
        """Per ghost Gauss point (panel, ring cell, h, g) two owner slots (owning panel,
        containing cell, 1-D weights, mass ratio, momentum matrix, share w: 1 and 0, or
        1/2 and 1/2 for a point on a cube edge); plus the ring cell list."""
        nr = lib().orc_ghost_count(self._h)
        n = 6 * nr * self.me * self.me * 2
        ring = np.empty(nr, np.int32)
        B, ic, jc = (np.empty(n, np.int32) for _ in range(3))
        wx, wy = np.empty((n, self.k)), np.empty((n, self.k))
        ratio, C, w = np.empty(n), np.empty((n, 4)), np.empty(n)
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        lib().orc_ghost_tables(self._h, ip(ring), ip(B), ip(ic), ip(jc), _p(wx), _p(wy), _p(ratio), _p(C), _p(w))
        return dict(ring=ring, B=B, ic=ic, jc=jc, wx=wx, wy=wy, ratio=ratio, C=C, w=w)

    def edge_tables(self):
        """Per (panel, side, cell, node): neighbour panel, side, cell, node and the B->A
        conversion (mass ratio, momentum matrix) at the shared edge point."""
        n = 6 * 4 * self.N * self.me
        B, sB, tB, gB = (np.empty(n, np.int32) for _ in range(4))
        ratio, C = np.empty(n), np.empty((n, 4))
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        lib().orc_edge_tables(self._h, ip(B), ip(sB), ip(tB), ip(gB), _p(ratio), _p(C))
        return dict(B=B, sideB=sB, tB=tB, gB=gB, ratio=ratio, C=C)

    def coriolis(self, panel, X, Y):
        return lib().orc_coriolis(self._h, int(panel), float(X), float(Y))

    def set_topography(self, sbar):
        """Bottom topography from cell averages of sqrtG phi_s, shape (6, N, N); None removes it."""
        if sbar is None:
            lib().orc_set_topography(self._h, None)
        else:
            sbar = _f64(sbar)
            assert sbar.shape == (6, self.N, self.N)
            lib().orc_set_topography(self._h, _p(sbar))

    def set_topography_case(self, case, params):
        """Analytic bottom surface (TOPO_*); initial conditions then read phi as phi_t."""
        P = _f64(list(params) + [0.0] * (4 - len(params)))
        lib().orc_set_topography_case(self._h, int(case), _p(P))

    def set_mountain(self, hs0=2000.0, R=np.pi / 9, lon_c=1.5 * np.pi, lat_c=np.pi / 6):
        """The isolated mountain of section 5.2 (eq. 5.8)."""
        self.set_topography_case(TOPO_MOUNTAIN, [hs0, R, lon_c, lat_c])

    def topography(self):
        out = np.empty((6, self.N, self.N))
        lib().orc_get_topography(self._h, _p(out))
        return out

    def set_topography_form(self, form):
        """0: total-geopotential form (eqs. 2.13-2.14, default); 1: depth form (2.1, 2.4)."""
        lib().orc_set_topography_form(self._h, int(form))

    def topo_psib(self, q):
        """The cell average of psi_B (eq. 2.14) alone, shape (2, 6, N, N)."""
        out = np.empty((2, 6, self.N, self.N))
        lib().orc_topo_psib(self._h, _p(_f64(q)), _p(out))
        return out

    def topography_point(self, panel, X, Y):
        return lib().orc_topography_point(self._h, int(panel), float(X), float(Y))

    def lmars_topo(self, direction, X, Y, qL, qR, sL, sR):
        F = np.empty(3)
        lib().orc_lmars_topo(self._h, int(direction), float(X), float(Y), _p(_f64(qL)), _p(_f64(qR)),
                             float(sL), float(sR), _p(F))
        return F

    def points(self):
        """Local unit-cell coordinates (xi, eta) of the n_poc reconstruction points."""
        g, _ = gauss(self.me)
        me = self.me
        xi = np.concatenate([np.full(me, -0.5), np.full(me, 0.5), g, g, np.tile(g, me)])
        eta = np.concatenate([g, g, np.full(me, -0.5), np.full(me, 0.5), np.repeat(g, me)])
        return xi, eta


def gauss(m):
    x = np.empty(m)
    w = np.empty(m)
    lib().orc_gauss(int(m), _p(x), _p(w))
    return x, w


def tpp_dweights_2d(k, xi, eta, direction):
    out = np.empty(k * k)
    lib().orc_tpp_dweights_2d(int(k), float(xi), float(eta), int(direction), _p(out))
    return out.reshape(k, k)


def sqrtg_grad(X, Y):
    out = np.empty(2)
    lib().orc_sqrtg_grad(float(X), float(Y), _p(out))
    return out


def weights_1d(n, o0, xi):
    out = np.empty(n)
    lib().orc_weights_1d(int(n), int(o0), float(xi), _p(out))
    return out


def tpp_weights_2d(k, xi, eta):
    out = np.empty(k * k)
    lib().orc_tpp_weights_2d(int(k), float(xi), float(eta), _p(out))
    return out.reshape(k, k)


def tpp_weights_2d_literal(k, xi, eta):
    out = np.empty(k * k)
    lib().orc_tpp_weights_2d_literal(int(k), float(xi), float(eta), _p(out))
    return out.reshape(k, k)


def weno_gamma(k, xi, eta):
    l = (k + 1) // 2
    g = np.empty(l * l)
    r = np.empty(1)
    lib().orc_weno_gamma(int(k), float(xi), float(eta), _p(g), _p(r))
    return g.reshape(l, l), float(r[0])


def weno1d_gamma(k, xi):
    g = np.empty((k + 1) // 2)
    r = np.empty(1)
    lib().orc_weno1d_gamma(int(k), float(xi), _p(g), _p(r))
    return g, float(r[0])


def weno1d_point(k, v, xi, eps=1e-40):
    return lib().orc_weno1d_point(int(k), _p(_f64(v)), float(xi), float(eps))


def weno_beta(l, o0x, o0y, Qsub):
    return lib().orc_weno_beta(int(l), int(o0x), int(o0y), _p(_f64(Qsub).ravel()))


def metric(X, Y):
    out = np.empty(7)
    lib().orc_metric(float(X), float(Y), _p(out))
    return out


def jacobian(panel, X, Y):
    out = np.empty(4)
    lib().orc_jacobian(int(panel), float(X), float(Y), _p(out))
    return out.reshape(2, 2)


def xyz(panel, X, Y):
    out = np.empty(3)
    lib().orc_xyz(int(panel), float(X), float(Y), _p(out))
    return out


def locate(p3):
    XY = np.empty(2)
    pan = lib().orc_locate(_p(_f64(p3)), _p(XY))
    return pan, XY
