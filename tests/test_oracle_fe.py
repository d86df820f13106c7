"""Pins of the oracle's conservative (bilinear finite-element) form of
Eqs. 6-7, an option beside the paper's finite differences of Eq. 7 (Sec. 2):
symmetry and definiteness of the volume-weighted operator, the discrete Gauss
law, the exact vacuum field of the sphere, and agreement with Eq. 7's
differences at second order."""
import numpy as np
import pytest

import oracle
from tests.inputs import ELECTRON, ION


def _cfg(n1, n2, alpha, fe=True, **kw):
    d = dict(alpha=alpha, x1_out=-0.1, phi_g=-1.5, phi_out=0.0, B=0.0, dt=0.1, n1=n1, n2=n2,
             species=[dict(ELECTRON, n_init=1000), dict(ION, n_init=1000)], no_inject=True, fe_operator=fe)
    d.update(kw)
    return d


def _interior(n1, n2, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n1 + 1, n2 + 1))
    u[0] = 0.0
    u[-1] = 0.0
    return u


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_volume_weighted_operator_is_symmetric_negative_definite(alpha):
    """u . (V L v) = v . (V L u) and u . (V L u) < 0 for functions that vanish
    on the Dirichlet rows; Eq. 7's differences are not symmetric (the
    contrast shows the test can fail)."""
    n1, n2 = 24, 16
    s = oracle.Sim(_cfg(n1, n2, alpha))
    V = s.grid("V")
    u, v = _interior(n1, n2, 1), _interior(n1, n2, 2)
    uLv, vLu = (u * V * s.apply_operator(v)).sum(), (v * V * s.apply_operator(u)).sum()
    assert abs(uLv - vLu) < 1e-12 * abs(uLv)
    assert (u * V * s.apply_operator(u)).sum() < 0 and (v * V * s.apply_operator(v)).sum() < 0
    fd = oracle.Sim(_cfg(n1, n2, alpha, fe=False))
    a, b = (u * V * fd.apply_operator(v)).sum(), (v * V * fd.apply_operator(u)).sum()
    assert abs(a - b) > 1e-6 * abs(a)


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_discrete_gauss_law(alpha):
    """The rows of the volume-weighted operator over all nodes sum to zero for
    any phi (the hat functions sum to one), so the net flux out of the
    grain and the outer surface equals the enclosed charge exactly: for the
    solution with charge rho, sum over the boundary rows of V L phi equals
    the charge sum(rho V) over the interior nodes."""
    n1, n2 = 24, 16
    s = oracle.Sim(_cfg(n1, n2, alpha))
    V = s.grid("V")
    phi = np.random.default_rng(3).standard_normal((n1 + 1, n2 + 1))
    total = (V * s.apply_operator(phi)).sum()
    assert abs(total) < 1e-12 * np.abs(V * s.apply_operator(phi)).sum()
    rho = 1.0 + np.random.default_rng(4).standard_normal((n1 + 1, n2 + 1))
    sol = s.solve(rho)
    VL = V * s.apply_operator(sol)
    assert np.abs(VL[1:-1] + (rho * V)[1:-1]).max() < 1e-10 * np.abs(rho * V).max()
    flux = VL[0].sum() + VL[-1].sum()
    assert flux == pytest.approx((rho * V)[1:-1].sum(), rel=1e-10)


@pytest.mark.parametrize("grid", [(16, 8), (48, 24)])
def test_sphere_vacuum_field_is_exact(grid):
    """For the sphere x1 = -1/r, where J g11 = 2 pi and J g12 = 0: the vacuum
    potential, linear in x1, is reproduced at every node on any grid (also by
    Eq. 7's differences)."""
    n1, n2 = grid
    s = oracle.Sim(_cfg(n1, n2, 0.0, phi_g=-2.0))
    phi = s.solve(np.zeros((n1 + 1, n2 + 1)))
    x1 = np.linspace(-1.0, -0.1, n1 + 1)[:, None]
    exact = -2.0 * (x1 - (-0.1)) / (-1.0 - (-0.1))
    assert np.abs(phi - exact).max() < 1e-12


def test_agrees_with_finite_differences_at_second_order():
    """The two discretisations of the same problem (smooth charge around a
    dipole grain) differ by O(h^2): the gap falls by about four per grid
    doubling."""
    gaps = []
    for n1, n2 in ((16, 16), (32, 32), (64, 64)):
        x1 = np.linspace(-1.0, -0.1, n1 + 1)[:, None]
        x2 = np.linspace(-1.0, 1.0, n2 + 1)[None, :]
        rho = np.exp(-((x1 + 0.6) / 0.2) ** 2) * (1.0 + 0.5 * x2)
        a = oracle.Sim(_cfg(n1, n2, 0.15)).solve(rho)
        b = oracle.Sim(_cfg(n1, n2, 0.15, fe=False)).solve(rho)
        gaps.append(np.abs(a - b).max())
    assert 3.0 < gaps[0] / gaps[1] < 5.5 and 3.0 < gaps[1] / gaps[2] < 5.5, gaps


def test_dipole_vacuum_field_convergence():
    """alpha != 0: the vacuum potential is still linear in x1 (x1 is harmonic),
    which Eq. 7's differences give exactly.  The linear field lies in the
    bilinear space, so the conservative form misses it only by its
    quadrature error: away from the axis that falls by sixteen per grid
    doubling, next to the poles (J growing like sqrt(1 - x2^2), handled by the
    t^2 placement of the points) by at least four."""
    inner, whole = [], []
    for n in (16, 32, 64):
        exact = -2.0 * (np.linspace(-1.0, -0.1, n + 1)[:, None] + 0.1) / (-0.9) * np.ones((1, n + 1))
        fe = oracle.Sim(_cfg(n, n, 0.2, phi_g=-2.0)).solve(np.zeros((n + 1, n + 1)))
        fd = oracle.Sim(_cfg(n, n, 0.2, fe=False, phi_g=-2.0)).solve(np.zeros((n + 1, n + 1)))
        assert np.abs(fd - exact).max() < 1e-12
        err = np.abs(fe - exact)
        inner.append(err[:, n // 4: 3 * n // 4 + 1].max())
        whole.append(err.max())
    assert whole[0] < 2e-5 * 2.0 and inner[0] > 1e-9
    assert inner[0] / inner[1] > 12.0 and inner[1] / inner[2] > 12.0, inner
    assert whole[0] / whole[1] > 3.5 and whole[1] / whole[2] > 3.5, whole
