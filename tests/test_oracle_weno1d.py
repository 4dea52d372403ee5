"""Pins of the oracle's dimension-by-dimension WENO-Z (the 1-D comparator of section 5.5,
fifth order), no GPU: the classic linear weights, exactness where every sub-stencil is
exact, convergence to the linear reconstruction on smooth data, non-oscillation at a
jump, the right-edge value against the textbook WENO-Z5 formula, the two-pass form in
2-D, and the finite-volume mass balance.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

OFFS = np.arange(-2, 3)


def _avg(f, c):
    x, w = O.gauss(8)
    return sum(w[q] * f(c + x[q]) for q in range(8))


@pytest.mark.parametrize("xi,want", [(0.5, ("1/10", "3/5", "3/10")), (-0.5, ("3/10", "3/5", "1/10")),
                                     (0.0, ("-9/80", "49/40", "-9/80"))])
def test_linear_weights_closed_forms(xi, want):
    """Fifth-order linear weights of the three 3-cell sub-stencils (left to right): the
    classic (1/10, 3/5, 3/10) at the right edge, mirrored at the left, and the negative
    (-9/80, 49/40, -9/80) at the centre (split by reading c2); exactly representable."""
    g, resid = O.weno1d_gamma(5, xi)
    np.testing.assert_allclose(g, [float(Fraction(w)) for w in want], rtol=0, atol=1e-14)
    assert resid < 1e-15


def test_exact_on_quadratics():
    """Every sub-stencil reproduces a quadratic and the split weights sum to one, so the
    nonlinear value is exact for any quadratic at any xi."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        c = rng.normal(size=3)
        v = [c[0] * 1.0 + c[1] * _avg(lambda x: x, o) + c[2] * _avg(lambda x: x * x, o) for o in OFFS]
        for xi in rng.uniform(-0.5, 0.5, 3):
            want = c[0] + c[1] * xi + c[2] * xi * xi
            assert abs(O.weno1d_point(5, v, xi) - want) < 1e-12 * (1 + np.abs(c).sum())


def test_smooth_data_converges_to_linear():
    """On smooth data the WENO-Z weights approach the linear ones fast enough that the
    nonlinear value departs from the fifth-order linear reconstruction far below the
    latter's own error (h = 0.1: 5e-10 against 2e-7), shrinking by >= 2^6 per halving."""
    dev = []
    for h in (0.2, 0.1, 0.05):
        def f(x, h=h):
            return np.sin(h * x + 0.3)
        v = np.array([_avg(f, c) for c in OFFS])
        lin = float(np.sum(O.weights_1d(5, -2, 0.5) * v))
        dev.append(abs(O.weno1d_point(5, v, 0.5) - lin))
        if h == 0.1:
            assert dev[-1] < 1e-2 * abs(lin - f(0.5))
    assert dev[0] / dev[1] > 64 and dev[1] / dev[2] > 64, dev


def test_non_oscillatory_at_a_jump():
    """At the edges of the cells next to a unit jump the linear fifth-order values
    overshoot (1.18) or undershoot (-0.18); the WENO-Z values stay in [0, 1]."""
    v = np.array([1.0, 1.0, 1.0, 0.0, 0.0])
    assert np.sum(O.weights_1d(5, -2, -0.5) * v) > 1.1
    for xi in (-0.5, 0.5, 0.0):
        assert -1e-12 <= O.weno1d_point(5, v, xi) <= 1.0 + 1e-12
    v = np.array([1.0, 1.0, 0.0, 0.0, 0.0])
    assert np.sum(O.weights_1d(5, -2, 0.5) * v) < -0.1
    assert abs(O.weno1d_point(5, v, 0.5)) < 1e-12


def test_two_pass_form_exact_on_biquadratics():
    """The 2-D comparator applies the 1-D scheme along x on each stencil row, then along y
    on the row values: for cell averages of X^a Y^b (a, b <= 2, X, Y in cell units) every
    pass is exact, so every point value of every cell is exact."""
    N, k = 8, 5
    o = O.Oracle(N, k, scheme=O.WENO1D)
    H, ne = o.H, N + 2 * o.H
    xi, eta = o.points()
    for a, b in [(0, 0), (1, 0), (0, 2), (2, 1), (2, 2)]:
        ext = np.zeros((3, 6, ne, ne))
        ax = np.array([_avg(lambda x: x ** a, c) for c in range(ne)])
        by = np.array([_avg(lambda y: y ** b, c) for c in range(ne)])
        ext[0] = np.outer(by, ax)[None]
        pts = o.reconstruct_all(ext)
        for j in (0, 3, N - 1):
            for i in (0, 5, N - 1):
                want = (i + H + xi) ** a * (j + H + eta) ** b
                np.testing.assert_allclose(pts[0, 2, j, i], want, rtol=1e-12, atol=1e-12)


def test_mass_conserved():
    """The comparator only changes the reconstruction: the finite-volume mass is kept to
    round-off (C8, three SSP-RK3 steps of a Rossby-Haurwitz wave)."""
    o = O.Oracle(8, 5, scheme=O.WENO1D)
    q = o.rossby_haurwitz()
    m0 = o.mass(q)
    q = o.step(q, 900.0, 3)
    assert abs(o.mass(q) - m0) / m0 < 5e-15
    assert np.isfinite(q).all()


def test_right_edge_is_textbook_weno_z5():
    """At xi = +1/2 every linear weight is positive, the split collapses to the plain
    combination, and the value is Borges et al.'s WENO-Z5: Jiang-Shu indicators in their
    closed forms, tau5 = |beta0 - beta2|, alpha = d (1 + tau5 / (beta + eps)) with
    d = (1/10, 3/5, 3/10), and the three third-order edge values."""
    rng = np.random.default_rng(5)
    eps = 1e-40
    for trial in range(30):
        v = rng.normal(size=5) * (10.0 if trial % 3 == 0 else 1.0)
        if trial % 5 == 0:
            v[3:] += 4.0  # a jump
        b0 = 13 / 12 * (v[0] - 2 * v[1] + v[2]) ** 2 + 0.25 * (v[0] - 4 * v[1] + 3 * v[2]) ** 2
        b1 = 13 / 12 * (v[1] - 2 * v[2] + v[3]) ** 2 + 0.25 * (v[1] - v[3]) ** 2
        b2 = 13 / 12 * (v[2] - 2 * v[3] + v[4]) ** 2 + 0.25 * (3 * v[2] - 4 * v[3] + v[4]) ** 2
        p = [(2 * v[0] - 7 * v[1] + 11 * v[2]) / 6, (-v[1] + 5 * v[2] + 2 * v[3]) / 6,
             (2 * v[2] + 5 * v[3] - v[4]) / 6]
        tau = abs(b0 - b2)
        alpha = [d * (1 + tau / (b + eps)) for d, b in zip((0.1, 0.6, 0.3), (b0, b1, b2))]
        want = sum(a * q for a, q in zip(alpha, p)) / sum(alpha)
        assert abs(O.weno1d_point(5, v, 0.5, eps) - want) < 1e-12 * (1 + np.abs(v).max()), trial
