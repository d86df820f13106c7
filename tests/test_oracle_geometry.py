"""Pins of the oracle's geometry (Eqs. 2-5, 8 and the metric of Eq. 10).

Each check compares the oracle with something other than itself: a closed
form, an identity of the mathematics, or brute force.
"""
import numpy as np
import pytest

import oracle

ALPHAS = [0.0, 0.1, 0.15, 0.225, -0.24]


@pytest.mark.parametrize("alpha", ALPHAS)
def test_round_trip_eq2_eq3(alpha):
    """Eq. 3 inverts Eq. 2 on the whole domain x1 in [-1, -0.02]."""
    rng = np.random.default_rng(7)
    for x1, x2 in zip(rng.uniform(-1.0, -0.02, 400), rng.uniform(-1.0, 1.0, 400)):
        r = oracle.r_of(alpha, x1, x2)
        assert r > 0
        assert abs(oracle.x1_of(alpha, r, x2) - x1) <= 1e-14 * max(1.0, abs(x1))


def test_sphere_reduction():
    """alpha = 0: x1 = -1/r, dA = 2 pi r^2 dx2, dOmega = 2 pi r^2 dr dx2 = 2 pi dx1 dx2 / x1^4."""
    for x1 in (-1.0, -0.5, -0.1):
        for x2 in (-1.0, -0.3, 0.0, 0.7, 1.0):
            assert oracle.r_of(0.0, x1, x2) == pytest.approx(-1.0 / x1, rel=1e-15)
            r = -1.0 / x1
            assert oracle.dA_dx2(0.0, x1, x2) == pytest.approx(2 * np.pi * r * r, rel=1e-14)
            assert oracle.dOmega(0.0, x1, x2) == pytest.approx(2 * np.pi / x1 ** 4, rel=1e-14)


def _x1x2_of_RZ(alpha, R, Z):
    r = np.hypot(R, Z)
    x2 = Z / r
    return oracle.x1_of(alpha, r, x2), x2


@pytest.mark.parametrize("alpha", ALPHAS)
def test_metric_matches_finite_differences(alpha):
    """The analytic d(x1,x2)/d(R,Z) agree with central differences of Eq. 2."""
    rng = np.random.default_rng(3)
    for _ in range(60):
        x1, x2 = rng.uniform(-0.95, -0.1), rng.uniform(-0.95, 0.95)
        r = oracle.r_of(alpha, x1, x2)
        R, Z = r * np.sqrt(1 - x2 * x2), r * x2
        m = oracle.metric(alpha, r, x2)
        h = 1e-6 * r
        a = np.array(_x1x2_of_RZ(alpha, R + h, Z)) - np.array(_x1x2_of_RZ(alpha, R - h, Z))
        b = np.array(_x1x2_of_RZ(alpha, R, Z + h)) - np.array(_x1x2_of_RZ(alpha, R, Z - h))
        fd = np.array([a[0], b[0], a[1], b[1]]) / (2 * h)
        assert np.allclose(m, fd, rtol=1e-6, atol=1e-8 / r ** 2)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_metric_reproduces_eq7_coefficients(alpha):
    """|grad x1|^2, grad x1 . grad x2 and |grad x2|^2 from the metric equal the
    coefficients printed in Eq. 7 (first, half the third, second)."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        x1, x2 = rng.uniform(-1.0, -0.05), rng.uniform(-1.0, 1.0)
        r = oracle.r_of(alpha, x1, x2)
        a, b, c, d = oracle.metric(alpha, r, x2)
        g11, g12, g22 = a * a + b * b, a * c + b * d, c * c + d * d
        s2 = 1 - x2 * x2
        assert g11 == pytest.approx(((r + 2 * alpha * x2) ** 2 + alpha ** 2 * s2) / r ** 6, rel=1e-12)
        assert 2 * g12 == pytest.approx(-2 * alpha * s2 / r ** 4, rel=1e-12, abs=1e-15)
        assert g22 == pytest.approx(s2 / r ** 2, rel=1e-12, abs=1e-15)


def _gl_integral(f, a, b, n_int=512):
    x, w = np.polynomial.legendre.leggauss(10)
    edges = np.linspace(a, b, n_int + 1)
    tot = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        xs = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
        tot += 0.5 * (hi - lo) * sum(wi * f(xi) for xi, wi in zip(xs, w))
    return tot


@pytest.mark.parametrize("alpha", [0.0, 0.15, 0.225, -0.24])
@pytest.mark.parametrize("x1", [-1.0, -0.4, -0.05])
def test_gauss_flux_of_harmonic_x1(alpha, x1):
    """x1 is (minus) the point-charge + dipole potential of Eq. 1, hence harmonic:
    the flux of grad x1 through every surface x1 = const is 4 pi R0.  Pins Eq. 4
    (surface element) together with the metric."""
    def f(x2):
        r = oracle.r_of(alpha, x1, x2)
        a, b, _, _ = oracle.metric(alpha, r, x2)
        return np.hypot(a, b) * oracle.dA_dx2(alpha, x1, x2)
    assert _gl_integral(f, -1.0, 1.0, 64) == pytest.approx(4 * np.pi, rel=1e-11)


@pytest.mark.parametrize("alpha", [0.0, 0.15, 0.225, -0.24])
def test_zero_vacuum_force_identity(alpha):
    """Surface integral of |grad x1| dx1/dZ dA vanishes on x1 = -1 (no net
    electrostatic force on a charged conductor in vacuum)."""
    def f(x2):
        r = oracle.r_of(alpha, -1.0, x2)
        a, b, _, _ = oracle.metric(alpha, r, x2)
        return np.hypot(a, b) * b * oracle.dA_dx2(alpha, -1.0, x2)
    scale = _gl_integral(lambda x2: abs(f(x2)), -1.0, 1.0, 64)
    assert abs(_gl_integral(f, -1.0, 1.0, 64)) < 1e-11 * scale


def _cube_integral_closed_form(alpha, x1):
    """Integral over x2 in [-1,1] of r(x1,x2)^3, in closed form: with
    u = sqrt(1 - 4 alpha x1 x2), r^3 dx2 = u (1+u)^3 du / (16 alpha x1^4)."""
    if alpha == 0.0:
        return -2.0 / x1 ** 3
    P = lambda u: u * u / 2 + u ** 3 + 0.75 * u ** 4 + u ** 5 / 5
    ua, ub = np.sqrt(1 - 4 * alpha * x1 * (-1.0)), np.sqrt(1 - 4 * alpha * x1 * 1.0)
    return (P(ub) - P(ua)) / (16 * alpha * x1 ** 4)


@pytest.mark.parametrize("alpha", [0.0, 0.15, 0.225, -0.24])
def test_node_volumes_sum_to_closed_form(alpha):
    """Sum of the hat-weighted node volumes (Eq. 5) equals the domain volume
    (2 pi / 3) int (r_out^3 - r_g^3) dx2, evaluated in closed form."""
    x1o = -0.05
    s = oracle.Sim(dict(alpha=alpha, x1_out=x1o, phi_g=0, phi_out=0, B=0, dt=0.1, n1=32, n2=16,
                        species=[dict(q=1, m=1, T=1, n_init=1000)], no_field=True))
    vol = 2 * np.pi / 3 * (_cube_integral_closed_form(alpha, x1o) - _cube_integral_closed_form(alpha, -1.0))
    # 8x8 Gauss-Legendre per cell of 1/x1^4-like integrands on a 32-cell grid
    # that reaches x1 = -0.05: quadrature error ~1e-12 relative.
    assert s.grid("V").sum() == pytest.approx(vol, rel=1e-10)
    assert s.scalars()["V_dom"] == pytest.approx(vol, rel=1e-12)
    if alpha == 0.0:
        assert vol == pytest.approx(4 * np.pi / 3 * (20.0 ** 3 - 1), rel=1e-14)
    assert (s.grid("V") > 0).all()


@pytest.mark.parametrize("alpha", [0.15, -0.24])
def test_monte_carlo_volume(alpha):
    """Brute force: the fraction of uniform points of a box that fall between
    the grain (Eq. 3 at x1 = -1) and the outer surface reproduces sum V_ij."""
    x1o = -0.25
    s = oracle.Sim(dict(alpha=alpha, x1_out=x1o, phi_g=0, phi_out=0, B=0, dt=0.1, n1=16, n2=8,
                        species=[dict(q=1, m=1, T=1, n_init=1000)], no_field=True))
    rng = np.random.default_rng(11)
    L = 6.0
    n = 400000
    p = rng.uniform(-L, L, (n, 3))
    r = np.linalg.norm(p, axis=1)
    x2 = p[:, 2] / r
    x1 = -(1.0 / r) * (1.0 + alpha * x2 / r)  # Eq. 2 evaluated independently of the oracle
    rg = np.array([oracle.r_of(alpha, -1.0, v) for v in x2[:2000]])
    assert (rg > 0).all()
    inside = (x1 >= -1.0) & (x1 <= x1o) & (r > 2 * abs(alpha))
    frac = inside.mean()
    vmc = frac * (2 * L) ** 3
    err = (2 * L) ** 3 * np.sqrt(frac * (1 - frac) / n)
    assert abs(vmc - s.grid("V").sum()) < 5 * err
    assert oracle.r_of(alpha, x1o, 1.0) < L and oracle.r_of(alpha, x1o, -1.0) < L


def test_gauss_legendre_exact_for_polynomials():
    x, w = oracle.gauss_legendre(8)
    for k in range(16):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert np.dot(w, x ** k) == pytest.approx(exact, abs=1e-14)
