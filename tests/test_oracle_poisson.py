"""Pins of the oracle's Poisson problem (Eqs. 6-7), node gradients and the
surface charge / electric force (Sec. 2 after Eq. 10)."""
import numpy as np
import pytest

import oracle
from tests.inputs import workload


def _sim(n1, n2, alpha, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, **kw):
    return oracle.Sim(workload(n1=n1, n2=n2, alpha=alpha, x1_out=x1_out, phi_g=phi_g, phi_out=phi_out,
                               n_init=1000, **kw))


def _node_x(n1, n2, x1_out):
    x1 = -1.0 + np.arange(n1 + 1) * ((x1_out + 1.0) / n1)
    x1[-1] = x1_out
    x2 = -1.0 + np.arange(n2 + 1) * (2.0 / n2)
    x2[-1] = 1.0
    return x1, x2


@pytest.mark.parametrize("alpha", [0.0, 0.15, 0.225, -0.24])
def test_laplace_exactness(alpha):
    """x1 is harmonic, so phi linear in x1 solves Eq. 6 with rho = 0; the
    second-order stencil reproduces it to rounding."""
    s = _sim(48, 24, alpha, x1_out=-0.05, phi_g=-3.0, phi_out=0.5)
    phi = s.solve(np.zeros((49, 25)))
    x1, _ = _node_x(48, 24, -0.05)
    exact = -3.0 + 3.5 * (x1 + 1.0) / 0.95
    assert np.abs(phi - exact[:, None]).max() < 1e-11


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_vacuum_capacitance_and_zero_force(alpha):
    """Vacuum: Q = 4 pi (phi_g - phi_out)/(1 + x1_out) (Gauss flux of the
    harmonic x1; the concentric-sphere capacitance at alpha = 0), and the
    electric force on the grain vanishes."""
    s = _sim(32, 64, alpha, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, no_inject=True)
    s.step(1)  # empty domain: deposit zero, solve, gradients, surface
    sc = s.scalars()
    Q0 = 4 * np.pi * (-2.5) / 0.9
    tol = 1e-12 if alpha == 0.0 else 2e-4
    assert sc["Q"] == pytest.approx(Q0, rel=tol)
    En, _, _ = s.surface()
    scale = 0.5 * np.mean(En ** 2) * 4 * np.pi
    assert abs(sc["FZ"]) < (1e-12 if alpha == 0.0 else 1e-3) * scale


def _manufactured(alpha, x1_out, smooth):
    """phi(x1, x2) vanishing-on-the-boundaries part plus the linear lift, and
    rho = -Laplacian(phi), the Laplacian taken in Cartesian coordinates of the
    x1(R, Z), x2(R, Z) of Eq. 2 -- independent of Eq. 7."""
    sp = pytest.importorskip("sympy")
    X, Z = sp.symbols("X Z", real=True)
    Y = sp.Symbol("Y", real=True)
    r = sp.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    x2 = Z / r
    x1 = -(1 / r) * (1 + alpha * x2 / r)
    pg, po = -2.5, 0.5
    if smooth == "quadratic":
        bump = 3.0 * (x1 + 1) * (x1 - x1_out) * (x2 + 0.5 * x2 ** 2)
    else:
        bump = 3.0 * (x1 + 1) * (x1 - x1_out) * sp.exp(2 * x1) * sp.sin(2 * x2 + 0.3)
    phi = pg + (po - pg) * (x1 + 1) / (x1_out + 1) + bump
    lap = sum(sp.diff(phi, v, 2) for v in (X, Y, Z))
    f_rho = sp.lambdify((X, Z), (-lap).subs(Y, 0), "numpy")
    f_phi = sp.lambdify((X, Z), phi.subs(Y, 0), "numpy")
    return f_phi, f_rho, pg, po


def _manufactured_errors(alpha, smooth, grids):
    x1_out = -0.2
    f_phi, f_rho, pg, po = _manufactured(alpha, x1_out, smooth)
    errs = []
    for n1, n2 in grids:
        x1, x2 = _node_x(n1, n2, x1_out)
        X1, X2 = np.meshgrid(x1, x2, indexing="ij")
        r = np.vectorize(lambda a, b: oracle.r_of(alpha, a, b))(X1, X2)
        R, Zc = r * np.sqrt(np.clip(1 - X2 ** 2, 0, None)), r * X2
        rho = np.asarray(f_rho(R, Zc), dtype=float) * np.ones_like(R)
        exact = np.asarray(f_phi(R, Zc), dtype=float) * np.ones_like(R)
        s = oracle.Sim(workload(n1=n1, n2=n2, alpha=alpha, x1_out=x1_out, phi_g=pg, phi_out=po, n_init=1000))
        phi = s.solve(rho)
        errs.append(np.abs(phi - exact).max())
    return np.array(errs)


@pytest.mark.parametrize("alpha", [0.0, 0.2, -0.24])
def test_manufactured_quadratic_is_exact(alpha):
    """Second-order differences (central, and one-sided at the poles) are exact
    on quadratics, so the discrete operator must reproduce the true 3-D
    Laplacian of phi = quadratic(x1) * quadratic(x2) exactly: every
    coefficient of Eq. 7 and every stencil weight is pinned to rounding."""
    errs = _manufactured_errors(alpha, "quadratic", ((16, 8), (32, 16)))
    assert errs.max() < 1e-11, errs


@pytest.mark.parametrize("alpha", [0.0, 0.2, -0.24])
def test_manufactured_solution_second_order(alpha):
    """Eq. 7 discretised to second order (Sec. 2): the error against a smooth
    transcendental exact solution falls by ~4 per grid halving."""
    errs = _manufactured_errors(alpha, "transcendental", ((16, 8), (32, 16), (64, 32)))
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[-1] < 1e-3
    assert (rates > 1.8).all(), (errs, rates)


def test_gradients_of_vacuum_solution():
    """Node gradients (central inside, one-sided second order on the edges) are
    exact on the linear-in-x1 vacuum solution: dphi/dx1 = dphi / (1 + x1_out)
    at every node, edges included, and dphi/dx2 = 0."""
    n1, n2, x1_out = 12, 10, -0.3
    s = _sim(n1, n2, 0.1, x1_out=x1_out, phi_g=-2.0, phi_out=1.0, no_inject=True)
    s.step(1)
    G1, G2 = s.grid("G1"), s.grid("G2")
    assert np.allclose(G1, 3.0 / (x1_out + 1.0), rtol=1e-10)
    assert np.abs(G2).max() < 1e-9


def test_solution_is_linear_in_rho_and_boundary():
    """Superposition: phi(rho_a + rho_b) = phi(rho_a) + phi(rho_b) - phi(0)."""
    s = _sim(24, 12, 0.15)
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal((2, 25, 13))
    pa, pb, pab, p0 = s.solve(a), s.solve(b), s.solve(a + b), s.solve(np.zeros_like(a))
    assert np.abs(pab - (pa + pb - p0)).max() < 1e-10 * np.abs(pab).max()
