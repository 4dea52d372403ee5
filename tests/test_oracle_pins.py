"""Pins of the oracle's building blocks against closed forms, exact arithmetic,
library routines and invariants (no GPU).

Each test names the passage of arXiv 2411.19185 whose content it fixes.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


# ---------------------------------------------------------------- quadrature
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 7])
def test_gauss_matches_numpy_and_is_exact(m):
    """Eqs. 3.5-3.6 use m_e-point Gauss-Legendre rules: equal to numpy's rule mapped
    to [-1/2, 1/2] and exact for degree <= 2m-1, not for degree 2m."""
    x, w = O.gauss(m)
    xr, wr = np.polynomial.legendre.leggauss(m)
    np.testing.assert_allclose(x, xr / 2, atol=1e-15)
    np.testing.assert_allclose(w, wr / 2, atol=1e-15)
    for d in range(2 * m):
        exact = 0.0 if d % 2 else 2 * 0.5 ** (d + 1) / (d + 1)
        assert abs(np.dot(w, x ** d) - exact) < 1e-15
    d = 2 * m
    exact = 2 * 0.5 ** (d + 1) / (d + 1)
    assert abs(np.dot(w, x ** d) - exact) > 1e-4 * exact


# ------------------------------------------------------- TPP weights (sec 3.1)
def _exact_weights_1d(n, o0, xi):
    """Exact rational solution of the 1-D cell-average system (textbook Gauss-Jordan
    over Fractions): r with sum_j r_j * avg_j(x^a) = xi^a for a < n."""
    xi = Fraction(xi)
    M = []
    for a in range(n):
        row = []
        for j in range(n):
            lo, hi = Fraction(2 * (o0 + j) - 1, 2), Fraction(2 * (o0 + j) + 1, 2)
            row.append((hi ** (a + 1) - lo ** (a + 1)) / (a + 1))
        row.append(xi ** a)
        M.append(row)
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[r][n] / M[r][r] for r in range(n)]


def test_weights_1d_closed_forms():
    """Section 3.1 in 1-D: the classic cell-average reconstruction weights at the
    right face, (-1/6, 5/6, 1/3) for k=3 and (1/30, -13/60, 47/60, 9/20, -1/20) for k=5."""
    np.testing.assert_allclose(O.weights_1d(3, -1, 0.5), [-1 / 6, 5 / 6, 1 / 3], atol=1e-15)
    np.testing.assert_allclose(O.weights_1d(5, -2, 0.5),
                               [1 / 30, -13 / 60, 47 / 60, 9 / 20, -1 / 20], atol=1e-15)


@pytest.mark.parametrize("k", [3, 5, 7, 9, 11])
@pytest.mark.parametrize("xi", [Fraction(1, 2), Fraction(-1, 2), Fraction(0), Fraction(3, 10)])
def test_weights_1d_exact_rational(k, xi):
    """Eqs. 3.11-3.15 in 1-D, solved exactly in rational arithmetic."""
    H = (k - 1) // 2
    ex = np.array([float(v) for v in _exact_weights_1d(k, -H, xi)])
    got = O.weights_1d(k, -H, float(xi))
    assert np.max(np.abs(got - ex)) < 2e-14 * max(1.0, np.max(np.abs(ex)))


@pytest.mark.parametrize("k", [3, 5])
def test_tpp_2d_kron_equals_literal_2d_solve(k):
    """Eq. 3.15 R = C A^-1 with the k^2 x k^2 monomial system equals the tensor
    product of 1-D weights (A and C factor for the tensor-product basis, eq. 3.7)."""
    for xi, eta in [(0.5, 0.1127), (-0.5, -0.3), (0.2, 0.4), (0.0, 0.0)]:
        a = O.tpp_weights_2d(k, xi, eta)
        b = O.tpp_weights_2d_literal(k, xi, eta)
        np.testing.assert_allclose(a, b, atol=1e-13)


def _cell_avg_monomial(a, c):
    """exact average of x^a over the unit cell centred at c"""
    return ((c + 0.5) ** (a + 1) - (c - 0.5) ** (a + 1)) / (a + 1)


@pytest.mark.parametrize("k", [3, 5, 7, 9, 11])
def test_tpp_reproduces_polynomials_to_degree_k_minus_1(k):
    """TPP of section 3.1 is exact for x^a y^b, a, b <= k-1, and not for x^k."""
    H = (k - 1) // 2
    o = O.Oracle(8 if k <= 7 else 12, k)
    xi, eta = o.points()
    offs = np.arange(-H, H + 1)
    for a, b in [(0, 0), (k - 1, 0), (0, k - 1), (k - 1, k - 1), (2, 1)]:
        if a > k - 1 or b > k - 1:
            continue
        st = np.outer([_cell_avg_monomial(b, c) for c in offs], [_cell_avg_monomial(a, c) for c in offs])
        for pt in range(o.npoc):
            R = O.tpp_weights_2d(k, xi[pt], eta[pt])
            val = np.sum(R * st)
            assert abs(val - xi[pt] ** a * eta[pt] ** b) < 1e-12 * (H + 1) ** (a + b)
    st = np.outer(np.ones(k), [_cell_avg_monomial(k, c) for c in offs])
    R = O.tpp_weights_2d(k, 0.5, 0.0)
    assert abs(np.sum(R * st) - 0.5 ** k) > 1e-6


# ---------------------------------------------------------- WENO (sec 3.2)
def test_weno5_gamma_tensor_product_closed_form():
    """Eq. 3.19: the least-squares linear weights have zero residual and equal the
    tensor product of the classic 1-D WENO5 weights: (1/10, 3/5, 3/10) at the right
    face and (-9/80, 49/40, -9/80) at the centre (negative: exercises eq. 3.20)."""
    g, res = O.weno_gamma(5, 0.5, 0.0)
    assert res < 1e-14
    ex = np.outer([-9 / 80, 49 / 40, -9 / 80], [1 / 10, 3 / 5, 3 / 10])
    np.testing.assert_allclose(g, ex, atol=1e-14)
    assert abs(g.sum() - 1) < 1e-14


@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_weno_gamma_sum_and_residual(k):
    """Eqs. 3.16-3.19 at every reconstruction point: zero residual, sum 1."""
    o = O.Oracle(12, k)
    xi, eta = o.points()
    for pt in range(o.npoc):
        g, res = O.weno_gamma(k, xi[pt], eta[pt])
        assert res < 1e-11
        assert abs(g.sum() - 1.0) < 1e-12


def test_weno_beta_closed_forms():
    """Eq. 3.25 as read (squared derivatives over the unit target cell): a constant
    gives 0, p = x gives 1, p = x^2 gives int(4x^2) + int(4) = 1/3 + 4, p = x*y gives
    int(y^2) + int(x^2) + int(1) = 1/12 + 1/12 + 1."""
    l = 3
    offs = np.arange(-1, 2)
    one = np.ones(l)
    lin = np.array([_cell_avg_monomial(1, c) for c in offs])
    sq = np.array([_cell_avg_monomial(2, c) for c in offs])
    assert abs(O.weno_beta(l, -1, -1, np.outer(one, one))) < 1e-14
    assert abs(O.weno_beta(l, -1, -1, np.outer(one, lin)) - 1.0) < 1e-13
    assert abs(O.weno_beta(l, -1, -1, np.outer(one, sq)) - (1 / 3 + 4)) < 1e-12
    assert abs(O.weno_beta(l, -1, -1, np.outer(lin, lin)) - (1 / 12 + 1 / 12 + 1)) < 1e-12
    # a shifted sub-stencil sees the same polynomial: same beta
    offs2 = np.arange(0, 3)
    sq2 = np.array([_cell_avg_monomial(2, c) for c in offs2])
    assert abs(O.weno_beta(l, 0, -1, np.outer(one, sq2)) - (1 / 3 + 4)) < 1e-12


@pytest.mark.parametrize("k", [3, 5, 9])
def test_weno_exact_on_substencil_polynomials(k):
    """Sub-stencil-space data (degree <= l-1 per variable): all betas are equal, tau
    is 0, the weights collapse to the linear ones and WENO is exact (sec 3.2)."""
    H, l = (k - 1) // 2, (k + 1) // 2
    o = O.Oracle(12, k, scheme=O.WENO)
    xi, eta = o.points()
    offs = np.arange(-H, H + 1)
    a, b = l - 1, 1
    st = np.outer([_cell_avg_monomial(b, c) for c in offs], [_cell_avg_monomial(a, c) for c in offs])
    st = st + 3.0
    for pt in range(o.npoc):
        val = o.weno_point(st, pt)
        assert abs(val - (xi[pt] ** a * eta[pt] ** b + 3.0)) < 1e-11


def test_weno_limits_a_jump_while_tpp_overshoots():
    """Non-oscillation (sec 3.2): at a step the TPP value overshoots the data range,
    the WENO value stays within it (up to a small tolerance)."""
    k = 5
    o = O.Oracle(12, k, scheme=O.WENO)
    st = np.ones((k, k))
    st[:, 3:] = 10.0
    xi, eta = o.points()
    tpp = [np.sum(O.tpp_weights_2d(k, xi[p], eta[p]) * st) for p in range(o.npoc)]
    weno = [o.weno_point(st, p) for p in range(o.npoc)]
    assert max(tpp) > 10.1 or min(tpp) < 0.9
    assert max(weno) < 10.0 + 1e-3 and min(weno) > 1.0 - 1e-3


# ---------------------------------------------------------- geometry (sec 2)
def _rand_points(n, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi / 4, np.pi / 4, size=(n, 2))


@pytest.mark.parametrize("p", range(6))
def test_jacobian_eq_2_10_matches_finite_differences(p):
    """J of eq. 2.10 equals r (cos(theta) dlambda/dx, cos(theta) dlambda/dy;
    dtheta/dx, dtheta/dy) computed by central differences of the point map."""
    for x, y in _rand_points(20, p):
        def ll(x_, y_):
            v = O.xyz(p, np.tan(x_), np.tan(y_))
            return np.arctan2(v[1], v[0]), np.arcsin(v[2])
        h = 1e-6
        l1, t1 = ll(x + h, y)
        l0, t0 = ll(x - h, y)
        l3, t3 = ll(x, y + h)
        l2, t2 = ll(x, y - h)
        wrap = lambda d: (d + np.pi) % (2 * np.pi) - np.pi
        lam, th = ll(x, y)
        Jfd = np.array([[np.cos(th) * wrap(l1 - l0), np.cos(th) * wrap(l3 - l2)],
                        [t1 - t0, t3 - t2]]) / (2 * h)
        J = O.jacobian(p, np.tan(x), np.tan(y))
        np.testing.assert_allclose(J, Jfd, atol=2e-8)


@pytest.mark.parametrize("p", range(6))
def test_metric_identities(p):
    """Eq. 2.12 J^T J = G_ij, and G^ij of eq. 2.6 (denominator (1+X^2)(1+Y^2)) is the
    inverse of eq. 2.7; sqrtG (eq. 2.8) = sqrt(det G_ij)."""
    for x, y in _rand_points(20, 10 + p):
        X, Y = np.tan(x), np.tan(y)
        m = O.metric(X, Y)
        Gup = np.array([[m[1], m[2]], [m[2], m[3]]])
        Glo = np.array([[m[4], m[5]], [m[5], m[6]]])
        J = O.jacobian(p, X, Y)
        np.testing.assert_allclose(J.T @ J, Glo, atol=1e-13)
        np.testing.assert_allclose(Gup @ Glo, np.eye(2), atol=1e-13)
        assert abs(m[0] - np.sqrt(np.linalg.det(Glo))) < 1e-13


def test_metric_pressure_identity():
    """d_x(sqrtG G^11) + d_y(sqrtG G^12) = 0 (and the same for the second row): the
    pressure flux of eq. 2.1 needs no metric source."""
    h = 1e-5
    for x, y in _rand_points(30, 3):
        f = lambda x_, y_: O.metric(np.tan(x_), np.tan(y_))
        a = (f(x + h, y)[0] * f(x + h, y)[1] - f(x - h, y)[0] * f(x - h, y)[1]) / (2 * h)
        b = (f(x, y + h)[0] * f(x, y + h)[2] - f(x, y - h)[0] * f(x, y - h)[2]) / (2 * h)
        c = (f(x + h, y)[0] * f(x + h, y)[2] - f(x - h, y)[0] * f(x - h, y)[2]) / (2 * h)
        d = (f(x, y + h)[0] * f(x, y + h)[3] - f(x, y - h)[0] * f(x, y - h)[3]) / (2 * h)
        assert abs(a + b) < 1e-8 and abs(c + d) < 1e-8


def test_sphere_area_and_panel_cover():
    """Sum over cells of <sqrtG> dx dy = 4 pi (unit sphere); every panel point maps
    back to its own panel."""
    o = O.Oracle(16, 5)
    sg = o.cell_sqrtg()
    assert abs(sg.sum() * o.dx ** 2 - 4 * np.pi) < 1e-9
    for p in range(6):
        for x, y in _rand_points(10, 20 + p) * 0.999:
            pan, XY = O.locate(O.xyz(p, np.tan(x), np.tan(y)))
            assert pan == p
            np.testing.assert_allclose(XY, [np.tan(x), np.tan(y)], atol=1e-13)


def test_sin_lat_eq_2_5_and_coriolis_sign():
    """f = 2 Omega sin(theta) with sin(theta) of eq. 2.5 and psi_C of eq. 2.3: at the
    north pole (centre of panel 5, sqrtG = 1, G^ij = I) x-momentum is turned towards
    -y (to the right of the motion, seen from above); at the south pole (panel 6)
    towards +y."""
    o = O.Oracle(8, 3)
    S = o.sources(4, 0.0, 0.0, [1.0, 1.0, 0.0])
    f = 2 * o.omega
    np.testing.assert_allclose(S, [0.0, 0.0, -f], atol=1e-20)
    S6 = o.sources(5, 0.0, 0.0, [1.0, 1.0, 0.0])
    np.testing.assert_allclose(S6, [0.0, 0.0, f], atol=1e-20)


# ----------------------------------------------------------- LMARS (sec 3.4)
def test_lmars_consistency_with_physical_flux():
    """With q_L = q_R the LMARS flux (eqs. 3.31-3.38) equals the analytic flux of
    eq. 2.16: (sqrtG phi u, sqrtG (phi u u + G^11 phi^2/2), sqrtG (phi u v + G^21 phi^2/2))."""
    o = O.Oracle(8, 3)
    rng = np.random.default_rng(5)
    for _ in range(20):
        X, Y = np.tan(rng.uniform(-0.78, 0.78, 2))
        m = O.metric(X, Y)
        phi = rng.uniform(5e3, 5e4)
        u, v = rng.uniform(-2e-5, 2e-5, 2)
        q = m[0] * phi * np.array([1.0, u, v])
        r2 = o.radius ** 2
        for d in (0, 1):
            F = o.lmars(d, X, Y, q, q)
            un = (u, v)[d]
            G1i = (m[1], m[2])[d] / r2
            G2i = (m[2], m[3])[d] / r2
            ex = np.array([q[0] * un, q[1] * un + 0.5 * m[0] * G1i * phi ** 2,
                           q[2] * un + 0.5 * m[0] * G2i * phi ** 2])
            np.testing.assert_allclose(F, ex, rtol=1e-12, atol=1e-12 * np.abs(ex).max())


def test_lmars_upwind_and_rest_state():
    """Fluid at rest with a phi jump: the mass flux is -(phi_R - phi_L)/(2c) scaled
    (flows from high to low phi); equal states at rest give zero mass flux."""
    o = O.Oracle(8, 3)
    m = O.metric(0.0, 0.0)
    qL = m[0] * np.array([2e4, 0.0, 0.0])
    qR = m[0] * np.array([1e4, 0.0, 0.0])
    F = o.lmars(0, 0.0, 0.0, qL, qR)
    assert F[0] > 0
    F0 = o.lmars(0, 0.0, 0.0, qL, qL)
    assert F0[0] == 0.0


def test_lmars_interface_velocity_identity_of_reading_c24():
    """Reading c24: eq. 3.32's (phi_R - phi_L) / (2 c) with c = (sqrt(phi_L) + sqrt(phi_R)) / 2
    (eqs. 3.34-3.35) equals sqrt(phi_R) - sqrt(phi_L), the form the library evaluates.  The
    oracle's mass flux (printed form) is reproduced from the identity form to round-off over
    random states, jumps of both signs included."""
    o = O.Oracle(8, 3)
    rng = np.random.default_rng(24)
    r2 = o.radius ** 2
    for _ in range(50):
        X, Y = np.tan(rng.uniform(-0.78, 0.78, 2))
        m = O.metric(X, Y)
        phiL, phiR = rng.uniform(1e3, 6e4, 2)
        uL, uR = rng.uniform(-3e-5, 3e-5, 2)
        vL, vR = rng.uniform(-3e-5, 3e-5, 2)
        qL = m[0] * phiL * np.array([1.0, uL, vL])
        qR = m[0] * phiR * np.array([1.0, uR, vR])
        for d in (0, 1):
            g = (m[1], m[3])[d] / r2  # G^ii
            sL, sR = np.sqrt(phiL), np.sqrt(phiR)
            upL, upR = (uL, vL)[d] / np.sqrt(g), (uR, vR)[d] / np.sqrt(g)
            ms = 0.5 * (upL + upR) - (sR - sL)
            mm = ms * np.sqrt(g)
            mass = 0.5 * (mm * (qL[0] + qR[0]) - abs(mm) * (qR[0] - qL[0]))
            F = o.lmars(d, X, Y, qL, qR)
            assert abs(F[0] - mass) <= 1e-12 * (abs(mm) * (qL[0] + qR[0]) + 1e-300)
