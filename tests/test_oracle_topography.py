"""Pins of the oracle's bottom-topography terms (no GPU): section 2's total-geopotential
form (eqs. 2.13-2.14), the LMARS pressure with phi_t (eq. 3.38) and the isolated
mountain of section 5.2 (eq. 5.8).

The checks are fixed by the mathematics, not by the oracle itself: the zero surface
reduces to the flat scheme bit for bit; the derivative weights differentiate
polynomials exactly; the sqrtG gradient matches finite differences of eq. 2.8; a
solid-body flow over a surface that is constant along its streamlines, with the
balanced free surface, is an exact steady state, as is a lake at rest over a hill, so
both residuals must fall at the design order.  On a copy of the oracle, a sign error
in psi_B, the pressure of eq. 3.38 taken with the depth instead of phi_t, a missing
-phi_t d(sqrtG) term or a missing 1/dx in the phi_t gradient each leave an O(1)
residual in one of these two states that does not fall with the grid spacing.
"""
import numpy as np
import pytest

from oracle import oracle as O

G = O.GRAVITY
H0_CASE5, U0_CASE5 = 5960.0, 20.0  # section 5.2


def _avg_monomial(a, c):
    """exact average of x^a over the unit cell centred at c"""
    return ((c + 0.5) ** (a + 1) - (c - 0.5) ** (a + 1)) / (a + 1)


def _lonlat_point(lam, th):
    p3 = np.array([np.cos(th) * np.cos(lam), np.cos(th) * np.sin(lam), np.sin(th)])
    pan, XY = O.locate(p3)
    return pan, XY[0], XY[1]


@pytest.mark.parametrize("k,scheme", [(3, O.TPP), (5, O.TPP), (5, O.WENO)])
def test_zero_surface_is_the_flat_scheme_bitwise(k, scheme):
    """With sqrtG phi_s = 0 the reconstructed sqrtG phi_t is sqrtG phi, phi_t = phi at every
    point and psi_B = 0, so the tendency equals the flat scheme's bit for bit."""
    o = O.Oracle(10, k, scheme=scheme)
    q = o.rossby_haurwitz()
    flat = o.tendency(q)
    o.set_topography(np.zeros((6, 10, 10)))
    assert np.array_equal(o.tendency(q), flat)
    o.set_topography(None)
    assert np.array_equal(o.tendency(q), flat)


def test_mountain_of_eq_5_8():
    """h_s = h_s0 (1 - r/R), r = min(R, distance in (lambda, theta)) with h_s0 = 2000 m,
    R = pi/9 and the centre at (3 pi/2, pi/6): 2000 m at the centre, 1000 m at half the
    radius, zero outside it.  The longitude difference is taken modulo 2 pi (reading c27),
    so the centre may be given as 3 pi/2 or -pi/2."""
    o = O.Oracle(8, 3)
    o.set_mountain()
    R, lc, tc = np.pi / 9, 1.5 * np.pi, np.pi / 6
    for lam, th, want in [(lc, tc, 2000.0), (lc, tc + R / 2, 1000.0), (lc + R / 2, tc, 1000.0),
                          (lc - 0.3 * R, tc - 0.4 * R, 1000.0), (lc, tc + 1.2 * R, 0.0),
                          (0.5 * np.pi, tc, 0.0), (-0.5 * np.pi, tc, 2000.0)]:
        pan, X, Y = _lonlat_point(lam, th)
        assert abs(o.topography_point(pan, X, Y) / G - want) < 1e-9 * 2000.0, (lam, th)


@pytest.mark.parametrize("k", [3, 5, 7])
def test_tpp_derivative_weights_are_exact_on_polynomials(k):
    """The derivative weights differentiate the TPP polynomial (the tensor form of eqs.
    3.7-3.15): for x^a y^b with a, b <= k-1 they give a x^(a-1) y^b and b x^a y^(b-1)
    at any point of the cell, from exact cell averages."""
    H = (k - 1) // 2
    offs = np.arange(-H, H + 1)
    rng = np.random.default_rng(3)
    for a, b in [(0, 0), (1, 0), (0, 1), (k - 1, 0), (0, k - 1), (k - 1, k - 1), (2, 1)]:
        if a > k - 1 or b > k - 1:
            continue
        st = np.outer([_avg_monomial(b, c) for c in offs], [_avg_monomial(a, c) for c in offs])
        for xi, eta in rng.uniform(-0.5, 0.5, size=(4, 2)):
            dx = np.sum(O.tpp_dweights_2d(k, xi, eta, 0) * st)
            dy = np.sum(O.tpp_dweights_2d(k, xi, eta, 1) * st)
            want_x = a * xi ** max(a - 1, 0) * eta ** b
            want_y = b * xi ** a * eta ** max(b - 1, 0)
            tol = 1e-11 * (H + 1) ** (a + b)
            assert abs(dx - want_x) < tol and abs(dy - want_y) < tol, (a, b, xi, eta)


def test_sqrtg_gradient_matches_finite_differences():
    """The closed-form gradient of eq. 2.8's sqrtG in the angles (x, y) agrees with
    centred differences of the metric routine to 1e-9."""
    h = 1e-5
    for x, y in [(0.1, -0.3), (-0.7, 0.7), (0.0, 0.0), (0.5, 0.2), (-0.78, -0.1)]:
        g = O.sqrtg_grad(np.tan(x), np.tan(y))
        fx = (O.metric(np.tan(x + h), np.tan(y))[0] - O.metric(np.tan(x - h), np.tan(y))[0]) / (2 * h)
        fy = (O.metric(np.tan(x), np.tan(y + h))[0] - O.metric(np.tan(x), np.tan(y - h))[0]) / (2 * h)
        assert abs(g[0] - fx) < 1e-9 and abs(g[1] - fy) < 1e-9, (x, y, g, fx, fy)


def test_lmars_lake_at_rest_across_a_step():
    """At rest with the same phi_t on both sides of a step in the bottom (different depths),
    LMARS of eqs. 3.32-3.38 with phi_t gives no mass flux and the pressure flux
    1/2 sqrtG G^{i1} phi_t^2 (reading c26)."""
    o = O.Oracle(8, 3)
    X, Y, pt = 0.3, -0.2, 5.0e4
    m = O.metric(X, Y)
    sG, r2 = m[0], O.RADIUS ** 2
    for d, (G1, G2) in enumerate([(m[1], m[2]), (m[2], m[3])]):
        phL, phR = 4.1e4, 3.3e4
        F = o.lmars_topo(d, X, Y, [sG * phL, 0, 0], [sG * phR, 0, 0], sG * (pt - phL), sG * (pt - phR))
        assert F[0] == 0.0
        np.testing.assert_allclose(F[1:], [0.5 * sG * G1 / r2 * pt ** 2, 0.5 * sG * G2 / r2 * pt ** 2],
                                   rtol=1e-14)


def test_initial_condition_reads_phi_as_total():
    """With an analytic surface set, an initial condition's phi is phi_t (reading c28, as in
    section 5.2 where h_0 is the free-surface height): depth + sqrtG phi_s averages equal the
    averages of the same field without topography, to round-off."""
    o = O.Oracle(12, 5)
    flat = o.geostrophic(u0=U0_CASE5, phi0=H0_CASE5 * G)
    o.set_mountain()
    q = o.geostrophic(u0=U0_CASE5, phi0=H0_CASE5 * G)
    s = o.topography()
    assert np.max(np.abs(q[0] + s - flat[0])) < 1e-11 * np.max(flat[0])
    assert np.max(s) > 0.5 * 2000.0 * G * np.max(o.cell_sqrtg())  # the mountain is resolved


def _rms_rates(make, k, Ns=(16, 32)):
    errs = []
    for N in Ns:
        o, q = make(N, k)
        d = o.tendency(q)
        errs.append([np.sqrt(np.mean(d[v] ** 2)) for v in range(3)])
    e = np.array(errs)
    return e, np.log2(e[0] / e[1])


@pytest.mark.parametrize("k", [3, 5])
def test_solid_body_flow_over_zonal_surface_is_steady(k):
    """u of eqs. 5.2-5.3 (alpha = pi/4, axis tilted with it, reading c21) over a surface
    h_s0 cos^2(theta') that is constant along the streamlines, with phi_t of eq. 5.1:
    div(phi u) = -u . grad(phi_s) = 0 and the momentum balance involves phi_t only, so the
    state is steady.  The discrete residual falls at about k - 1 (the phi_t gradient in
    psi_B loses one order) in every variable."""
    def make(N, k):
        o = O.Oracle(N, k, coriolis_tilt=np.pi / 4)
        o.set_topography_case(O.TOPO_ZONAL, [2000.0, np.pi / 4])
        return o, o.geostrophic(alpha=np.pi / 4, u0=U0_CASE5, phi0=H0_CASE5 * G)
    e, rate = _rms_rates(make, k)
    assert np.all(rate > k - 1.2), (e, rate)


@pytest.mark.parametrize("k,scheme", [(3, O.TPP), (5, O.TPP), (5, O.WENO)])
def test_lake_at_rest_over_a_hill(k, scheme):
    """phi_t constant, u = 0, over a Gaussian hill of 2000 m: reconstructing sqrtG phi_t
    (the purpose of eq. 2.13) leaves only the truncation error of reconstructing sqrtG
    times a constant, which falls at about the design order in every variable -- also
    with the genuine-2D WENO-Z, whose nonlinear weights then see a smooth sqrtG phi_t
    instead of the bottom's imprint on the depth."""
    def make(N, k):
        o = O.Oracle(N, k, scheme=scheme)
        o.set_topography_case(O.TOPO_HILL, [2000.0, np.pi / 9, 1.5 * np.pi, np.pi / 6])
        return o, o.geostrophic(u0=0.0, phi0=H0_CASE5 * G)
    e, rate = _rms_rates(make, k)
    assert np.all(rate > k - 1.0), (e, rate)


@pytest.mark.parametrize("k,scheme", [(3, O.TPP), (5, O.WENO)])
def test_mass_conserved_over_the_mountain(k, scheme):
    """Section 5.2's flow over the isolated mountain keeps the finite-volume mass
    (the depth's integral) to round-off: psi_B has no mass component and the mass flux
    is still computed once per shared edge."""
    o = O.Oracle(10, k, scheme=scheme)
    o.set_mountain()
    q = o.geostrophic(u0=U0_CASE5, phi0=H0_CASE5 * G)
    m0 = o.mass(q)
    q = o.step(q, 900.0, 3)
    assert abs(o.mass(q) - m0) / m0 < 5e-15


def test_total_form_keeps_a_lake_at_rest_over_the_cone_the_depth_form_does_not():
    """Section 2's reason for eq. 2.13: over the mountain of eq. 5.8 (kinks at its rim and
    top) a lake at rest stays at rest to the truncation error of a constant phi_t in the
    total-geopotential form -- the residual falls at the design order -- while the depth
    form of eqs. 2.1 and 2.4 reconstructs the kinked depth and its residual barely falls
    with the grid (k = 5: more than 3000 times larger at C32)."""
    res = {}
    for form in (0, 1):
        for N in (16, 32):
            o = O.Oracle(N, 5)
            o.set_mountain()
            o.set_topography_form(form)
            d = o.tendency(o.geostrophic(u0=0.0, phi0=H0_CASE5 * G))
            res[form, N] = np.array([np.sqrt(np.mean(d[v] ** 2)) for v in range(3)])
    assert np.all(np.log2(res[0, 16] / res[0, 32]) > 4.0), res
    assert np.all(np.log2(res[1, 16] / res[1, 32]) < 1.0), res
    assert np.all(res[1, 32] > 1e3 * res[0, 32]), res
