"""Pins of the oracle's Boltzmann-electron option (electrons not simulated,
n_e = exp(phi) in Eq. 6, the option Sec. 2 mentions): the Debye-Hueckel
limit of a charged sphere in a uniform ion background, the fixed point of the
linear solve, the discrete maximum principle, and an ion-only run."""
import numpy as np
import pytest

import oracle
from tests.inputs import ION


def _cfg(n1, n2, alpha=0.0, phi_g=-1.0, **kw):
    d = dict(alpha=alpha, x1_out=-0.1, phi_g=phi_g, phi_out=0.0, B=0.0, dt=1.0, n1=n1, n2=n2,
             species=[dict(ION, n_init=20000)], no_inject=True, boltzmann=True)
    d.update(kw)
    return d


def _debye_hueckel(r, eps, r_out):
    """Delta phi = phi around a unit sphere at potential eps inside a grounded
    shell at r_out: phi = eps sinh(r_out - r) / (r sinh(r_out - 1))."""
    return eps * np.sinh(r_out - r) / (r * np.sinh(r_out - 1.0))


def _radii(n1, n2):
    x1 = np.linspace(-1.0, -0.1, n1 + 1)
    return np.array([[oracle.r_of(0.0, a, b) for b in np.linspace(-1, 1, n2 + 1)] for a in x1])


def test_debye_hueckel_limit_second_order():
    """A weakly charged sphere (phi_g = 1e-6) in a uniform ion background
    (rho_i = 1 = n0): exp(phi) - 1 = phi to 1e-6 relative, so the solution is
    the screened Yukawa potential of the sphere in its shell; the discrete
    solution converges to it at second order in h."""
    eps = 1e-6
    errs = []
    for n1 in (32, 64, 128):
        s = oracle.Sim(_cfg(n1, 8, phi_g=eps))
        phi = s.solve(np.ones((n1 + 1, 9)))
        r = _radii(n1, 8)
        r_out = r[-1, 0]
        errs.append(np.abs(phi - _debye_hueckel(r, eps, r_out)).max() / eps)
    assert errs[2] < 2e-3, errs
    assert 3.2 < errs[0] / errs[1] < 4.8 and 3.2 < errs[1] / errs[2] < 4.8, errs


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_solution_is_a_fixed_point_of_the_linear_solve(alpha):
    """With the ions of a volume load and a strongly negative grain, the Newton
    solution phi reproduces itself through the linear solve of Eqs. 6-7 with
    the total charge rho_i - exp(phi)."""
    s = oracle.Sim(_cfg(48, 24, alpha=alpha, phi_g=-2.5))
    s.load_volume(0, 20000)
    s.deposit()
    rho_i = s.grid("rho")
    phi = s.solve(rho_i)
    back = s.solve_linear(rho_i - np.exp(phi))
    assert np.abs(back - phi).max() < 1e-11
    assert np.abs(phi[0] + 2.5).max() == 0.0 and np.abs(phi[-1]).max() == 0.0


def test_screening_bounds():
    """Uniform ions, negative grain: the net charge is positive wherever
    phi < 0, so the discrete maximum principle bounds the potential between
    the vacuum potential and zero, strictly inside."""
    s = oracle.Sim(_cfg(64, 16, phi_g=-3.0))
    ones = np.ones((65, 17))
    phi = s.solve(ones)
    vac = s.solve_linear(np.zeros((65, 17)))
    inner = phi[1:-1]
    assert (inner > vac[1:-1]).all() and (inner < 0).all()
    # the screened potential decays much faster than the vacuum one: a few
    # Debye lengths out (node 53: r = 3.9) it is a tenth of it
    assert abs(phi[53, 8]) < 0.15 * abs(vac[53, 8])


def test_ion_only_run():
    """Ten steps with Boltzmann electrons and one pushed species: the
    warm-started Newton takes a few iterations, the tallies are finite and the
    electron-free bookkeeping closes."""
    cfg = _cfg(32, 16, alpha=0.15, phi_g=-2.5, dt=0.5)
    cfg.pop("no_inject")
    s = oracle.Sim(cfg)
    s.load_volume(0, 20000)
    s.step(10)
    h = s.history()
    assert h.shape == (10, 11) and np.isfinite(h).all()
    assert 1 <= s.newton_iterations() <= 6
    c = s.counts()[0]
    assert c["loaded"] + c["injected"] == c["absorbed"] + c["escaped"] + c["resident"]
    assert c["absorbed"] > 0


def test_boltzmann_rejects_field_free_and_isolated_grain():
    with pytest.raises(ValueError):
        oracle.Sim(_cfg(32, 16, no_field=True))
    with pytest.raises(ValueError):
        oracle.Sim(_cfg(32, 16, floating=True))


@pytest.mark.parametrize("phi_g", [-2.5, -0.5])
def test_boltzmann_electron_current(phi_g):
    """The grain collects the Boltzmann electrons' one-sided Maxwellian flux,
    n0 exp(phi_g) sqrt(Te / 2 pi me) per unit area: with no ions the grain
    current of a unit sphere (area 4 pi) is -4 pi exp(phi_g) / sqrt(2 pi) every
    step."""
    s = oracle.Sim(_cfg(32, 16, phi_g=phi_g))
    s.step(3)
    h = s.history()
    assert np.allclose(h[:, 1], -4 * np.pi * np.exp(phi_g) / np.sqrt(2 * np.pi), rtol=1e-12, atol=0)
