"""Pins of the oracle's perturbed-jet initial condition (section 5.4, eqs. 5.16-5.18,
Galewsky et al. 2004), no GPU: the balance integral against an independent
arbitrary-precision quadrature, its derivative against the balance it encodes, the jet
and bump closed forms, the mean depth of reading c30, and the steadiness of the
unperturbed jet under the scheme.
"""
import numpy as np
import pytest

from oracle import oracle as O

P7 = list(O.GALEWSKY)  # umax, theta0, theta1, theta2, alpha, beta, hhat
TH0, TH1, TH2 = P7[1], P7[2], P7[3]


def _phi_u(o, lam, th, hhat=0.0, phi0=1.0):
    P = P7[:6] + [hhat, phi0]
    return o.ic_point(O.IC_GALEWSKY, P, lam, th)


def test_jet_profile_eq_5_16():
    """u = umax at the jet centre (there (theta - theta0)(theta - theta1) = -(dtheta/2)^2, so
    the exponential equals e_n), zero outside (theta0, theta1), and no meridional wind."""
    o = O.Oracle(8, 3)
    mid = 0.5 * (TH0 + TH1)
    assert abs(_phi_u(o, 0.4, mid)[1] - 80.0) < 1e-12 * 80.0
    for th in (TH0 - 0.01, TH0, TH1, TH1 + 0.2, -0.7):
        assert _phi_u(o, 0.4, th)[1] == 0.0
    assert _phi_u(o, 0.4, mid)[2] == 0.0


def test_balance_integral_matches_arbitrary_precision_quadrature():
    """phi0 - phi of the unperturbed jet is the integral of eq. 5.17; mpmath's adaptive
    tanh-sinh quadrature at 30 digits gives the same value to 1e-13."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    o = O.Oracle(8, 3)
    a, Om = O.RADIUS, O.OMEGA
    en = mp.e ** (-4 / (mp.mpf(TH1) - TH0) ** 2)

    def u(t):
        return 0 if (t <= TH0 or t >= TH1) else P7[0] / en * mp.e ** (1 / ((t - TH0) * (t - TH1)))

    for th in (TH0 + 0.1, 0.5 * (TH0 + TH1), TH1 - 0.05, TH1, 1.3):
        want = mp.quad(lambda t: a * u(t) * (2 * Om * mp.sin(t) + mp.tan(t) * u(t) / a),
                       [TH0, 0.5 * (TH0 + TH1), min(th, TH1)])
        got = 1.0 - _phi_u(o, 0.3, th)[0]
        assert abs(got - float(want)) < 1e-13 * abs(float(want)), th
    assert _phi_u(o, 0.3, TH0 - 0.2)[0] == 1.0


def test_balance_is_gradient_wind():
    """Differentiating eq. 5.17: d phi / d theta = -a u (f + tan(theta) u / a), the
    gradient-wind balance of the zonal jet (fourth-order centred differences: 1e-7
    relative, with an absolute floor of 1e-7 m^2/s^2 per radian on the jet's flanks, where
    the difference quotient's rounding exceeds the relative bound)."""
    o = O.Oracle(8, 3)
    a, Om, h = O.RADIUS, O.OMEGA, 2e-4

    def f(t):
        return _phi_u(o, 0.0, t)[0]

    for th in (0.5, 0.7, 0.8, 0.95, 1.05):
        dphi = (-f(th + 2 * h) + 8 * f(th + h) - 8 * f(th - h) + f(th - 2 * h)) / (12 * h)
        u = _phi_u(o, 0.0, th)[1]
        want = -a * u * (2 * Om * np.sin(th) + np.tan(th) * u / a)
        assert abs(dphi - want) < 1e-7 * max(abs(want), 1.0), th


def test_perturbation_eq_5_18():
    """phi' = g hhat cos(theta) exp(-(lambda/alpha)^2 - ((theta2 - theta)/beta)^2)."""
    o = O.Oracle(8, 3)
    g = O.GRAVITY
    for lam, th in ((0.0, TH2), (0.2, TH2), (-0.1, TH2 + 0.05), (2.5, 0.3)):
        d = _phi_u(o, lam, th, hhat=120.0)[0] - _phi_u(o, lam, th)[0]
        want = g * 120.0 * np.cos(th) * np.exp(-(lam / P7[4]) ** 2 - ((TH2 - th) / P7[5]) ** 2)
        assert abs(d - want) < 1e-9 * g * 120.0, (lam, th)


def test_mean_depth_is_10_km():
    """Reading c30 (phi0 = 0 asks for Galewsky's constant): the area mean of phi over the
    unperturbed state's cell averages is g x 10 km to 1e-10."""
    o = O.Oracle(24, 5)
    q = o.galewsky(perturbed=False)
    mean = q[0].sum() / o.cell_sqrtg().sum()
    assert abs(mean / (O.GRAVITY * 1e4) - 1.0) < 1e-10


@pytest.mark.parametrize("k", [3, 5])
def test_unperturbed_jet_is_steady(k):
    """Without phi' the balanced zonal jet is a steady solution; the scheme's tendency falls
    at close to the design order (C32 -> C64)."""
    errs = []
    for N in (32, 64):
        o = O.Oracle(N, k)
        q = o.galewsky(perturbed=False)
        d = o.tendency(q)
        errs.append([np.sqrt(np.mean(d[v] ** 2)) / np.sqrt(np.mean(q[v] ** 2)) for v in range(3)])
    e = np.array(errs)
    rate = np.log2(e[0] / e[1])
    assert np.all(rate > k - 1.2), (e, rate)
