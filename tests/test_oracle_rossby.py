"""Pin of the oracle's Rossby-Haurwitz initial condition (section 5.3, eqs. 5.10-5.15)
against the property that defines its geopotential (no GPU).

The wind of eqs. 5.11-5.12 is non-divergent.  The geopotential of eqs. 5.10 and
5.13-5.15 is the one that keeps it so at t = 0: taking the divergence of the momentum
equation in vector-invariant form, dv/dt + (f + zeta) k x v + grad(Phi + |v|^2/2) = 0,
the divergence tendency vanishes exactly when

    lap(Phi + |v|^2/2) + div((f + zeta) k x v) = 0.

The test evaluates the oracle's point values (Phi, u, v) on small longitude-latitude
stencils, forms both terms with fourth-order central differences in spherical
coordinates, and checks that their sum vanishes separately in the zonal mean (A(theta),
eq. 5.13), in the wavenumber-R harmonic (B, eq. 5.14) and in the wavenumber-2R harmonic
(C, eq. 5.15), each relative to the same harmonic of lap Phi.  Only C contributes to the
2R harmonic of lap Phi, only B to the R one, so a factor (1 + d) on C, B or A leaves a
relative residual d in its harmonic: a dropped term, a wrong sign or a wrong factor fails.
The steady geostrophic flow of eqs. 5.1-5.3 satisfies the same balance and checks the
finite-difference machinery.
"""
import numpy as np
import pytest

from oracle import oracle as O

D = 1e-3  # finite-difference step (radians)
M = 6     # stencil half-width: (2M+1)^2 point values per evaluation


def _d(f, axis):
    """Fourth-order central first difference along an axis (two samples lost at each end)."""
    n = f.shape[axis]
    t = lambda s: np.take(f, range(s, n - 4 + s), axis=axis)  # noqa: E731
    return (t(0) - 8.0 * t(1) + 8.0 * t(3) - t(4)) / (12.0 * D)


def _c(f, k):
    """Drop k samples at each end of both axes."""
    return f[k:f.shape[0] - k, k:f.shape[1] - k]


def balance_terms(o, case, params, lam0, th0):
    """(residual, lap Phi) of the divergence-tendency balance at (lam0, th0)."""
    lam = lam0 + D * np.arange(-M, M + 1)
    th = th0 + D * np.arange(-M, M + 1)
    Phi, U, V = (np.empty((2 * M + 1, 2 * M + 1)) for _ in range(3))  # [theta][lambda]
    for j, t in enumerate(th):
        for i, l in enumerate(lam):
            Phi[j, i], U[j, i], V[j, i] = o.ic_point(case, params, l, t)
    a, Om = o.radius, o.omega
    ct = np.repeat(np.cos(th)[:, None], 2 * M + 1, axis=1)
    f = 2 * Om * np.repeat(np.sin(th)[:, None], 2 * M + 1, axis=1)
    # relative vorticity (dV/dlam - d(U cos)/dtheta) / (a cos) on the inner 9 x 9
    zeta = (_d(V, 1)[2:-2, :] - _d(U * ct, 0)[:, 2:-2]) / (a * _c(ct, 2))
    # div((f + zeta) k x v) with k x v = (-V, U), on the inner 5 x 5
    absv = _c(f, 2) + zeta
    Al, At = -absv * _c(V, 2), absv * _c(U, 2)
    div = (_d(Al, 1)[2:-2, :] + _d(At * _c(ct, 2), 0)[:, 2:-2]) / (a * _c(ct, 4))

    def lap(F):  # spherical Laplacian on the inner 5 x 5
        Fll = _d(_d(F, 1), 1)[4:-4, :]
        Ftt = _d(_d(F, 0) * ct[2:-2, :], 0)[:, 4:-4]
        c5 = _c(ct, 4)
        return Fll / (a * a * c5 * c5) + Ftt / (a * a * c5)

    lP = lap(Phi)
    res = lap(Phi + 0.5 * (U * U + V * V)) + div
    return res[2, 2], lP[2, 2]


def _ring(o, case, params, th0, n=32):
    """Longitude harmonics of the residual and of lap Phi along the circle theta = th0."""
    r, lp = np.empty(n), np.empty(n)
    for t in range(n):
        r[t], lp[t] = balance_terms(o, case, params, 2 * np.pi * t / n + 0.05, th0)
    return np.fft.rfft(r) / n, np.fft.rfft(lp) / n


@pytest.fixture(scope="module")
def orc():
    O.build_oracle()
    return O.Oracle(4, 3)


RH = [7.848e-6, 7.848e-6, 4.0, 8000.0]  # omega, K, R, h0 of section 5.3


@pytest.mark.parametrize("th0", [-0.9, -0.35, 0.2, 0.6, 0.95])
def test_rossby_haurwitz_geopotential_keeps_the_wind_non_divergent(orc, th0):
    """Eqs. 5.10-5.15: the divergence tendency of the Rossby-Haurwitz state vanishes in
    each of the longitude harmonics 0, R and 2R separately (relative to the same harmonic
    of lap Phi, itself a sizeable part of the field), and nothing is left elsewhere."""
    rh, lh = _ring(orc, O.IC_ROSSBY, RH, th0)
    R = int(RH[2])
    scale = np.max(np.abs(lh))
    for mode in (0, R, 2 * R):
        assert abs(lh[mode]) > 1e-3 * scale, (th0, mode)
        assert abs(rh[mode]) < 1e-6 * abs(lh[mode]), (th0, mode, abs(rh[mode]), abs(lh[mode]))
    assert np.max(np.abs(rh)) < 1e-6 * scale


@pytest.mark.parametrize("th0", [-0.9, 0.3, 1.1])
def test_geostrophic_state_satisfies_the_same_balance(orc, th0):
    """Eqs. 5.1-5.3 with alpha = 0 (f = 2 Omega sin theta): a steady state, so its
    divergence tendency vanishes as well; checks the difference operators."""
    u0 = 2 * np.pi * orc.radius / (12 * 86400.0)
    for lam0 in (0.1, 1.7, -2.3):
        r, lp = balance_terms(orc, O.IC_GEOSTROPHIC, [0.0, u0, 2.94e4], lam0, th0)
        assert abs(r) < 1e-6 * abs(lp), (th0, lam0, r, lp)
