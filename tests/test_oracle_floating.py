"""Pins of the oracle's isolated-grain option (the grain potential follows the
charge it collects; the paper itself holds phi_g fixed, Sec. 1).  The
electrostatics of a charged conducting sphere inside a grounded spherical
shell fixes what the option must give; superposition and charge bookkeeping
fix the rest."""
import numpy as np
import pytest

import oracle
from tests.inputs import ELECTRON, ION, workload


def _vacuum_cfg(n1, n2, phi_g, **kw):
    d = dict(alpha=0.0, x1_out=-0.1, phi_g=phi_g, phi_out=0.0, B=0.0, dt=0.1, n1=n1, n2=n2,
             species=[dict(ELECTRON, n_init=10000), dict(ION, n_init=10000)], no_inject=True,
             floating=True)
    d.update(kw)
    return d


def _ions_falling_in(n, r0, v0, seed):
    """n ions on the sphere r = r0 at random polar angles, moving radially
    inwards at speed v0 (logical positions, cylindrical velocities)."""
    rng = np.random.default_rng(seed)
    x2 = rng.uniform(-0.95, 0.95, n)
    R, Z = r0 * np.sqrt(1 - x2 * x2), r0 * x2
    x1 = np.array([oracle.x1_of(0.0, r0, c) for c in x2])
    return np.column_stack([x1, x2, -v0 * R / r0, -v0 * Z / r0, np.zeros(n)])


def _sphere_capacitance(x1_out):
    """C = 4 pi eps0 / (1/r_g - 1/r_out) of a unit sphere inside a concentric
    grounded shell (eps0 = 1, r_g = 1)."""
    r_out = oracle.r_of(0.0, x1_out, 0.3)
    return 4 * np.pi / (1.0 - 1.0 / r_out)


@pytest.mark.parametrize("grid", [(32, 16), (64, 32)])
def test_vacuum_grain_charge_is_the_shell_capacitance(grid):
    """No particles: the first step fixes the grain charge at C phi_g, with C
    the capacitance of the sphere in its grounded shell.  For alpha = 0 the
    coordinate x1 of Eq. 2 is -1/r, in which the vacuum potential is linear, so
    the second-order differences (and the one-sided surface derivative)
    reproduce it, and C, to rounding on any grid.  With nothing collected the
    potential then stays at phi_g."""
    phi_g = -1.7
    s = oracle.Sim(_vacuum_cfg(*grid, phi_g))
    s.step(3)
    h = s.history()
    C = _sphere_capacitance(-0.1)
    assert h[0, 6] == pytest.approx(C * phi_g, rel=1e-12)
    assert np.allclose(h[:, 10], phi_g, rtol=0, atol=1e-12)
    assert np.allclose(h[:, 6], h[0, 6], rtol=1e-13, atol=0)


def test_collected_charge_raises_the_potential():
    """Ions falling onto an isolated sphere: while they approach, the grain
    keeps its charge (its potential moves instead); once they are absorbed the
    grain charge has grown by the ions' charge N q w and, the domain being
    empty again, the potential has risen by N q w / C, C the capacitance of
    the sphere in its shell."""
    phi_g = -1.0
    s = oracle.Sim(_vacuum_cfg(64, 32, phi_g))
    s.step(1)
    Q0 = s.history()[0, 6]
    n = 300
    s.add_particles(1, _ions_falling_in(n, 1.05, 2.0, seed=4))
    s.step(1)  # the ions are deposited, then absorbed by the push
    assert s.counts()[1]["absorbed"] == n
    s.step(1)
    h = s.history()
    w = s.scalars()["w1"]
    dq = n * 1.0 * w
    assert h[1, 6] == pytest.approx(Q0, rel=1e-12)           # charge conserved while they approach
    assert h[1, 10] != pytest.approx(phi_g, rel=1e-6)        # ... the potential moved
    assert h[1, 1] * 0.1 == pytest.approx(dq, rel=1e-12)     # current of the step
    assert h[2, 6] == pytest.approx(Q0 + dq, rel=1e-12)
    assert h[2, 10] - phi_g == pytest.approx(dq / _sphere_capacitance(-0.1), rel=1e-9)


def test_floating_first_step_equals_fixed_potential():
    """Superposition: the first step of an isolated grain (phi_0 + phi_g phi_vac)
    is the fixed-potential step (one direct solve with the grain at phi_g)."""
    base = workload(n1=32, n2=16, alpha=0.15, B=0.5, n_init=20000, seed=3, phi_g=-1.3)
    a, b = oracle.Sim(base), oracle.Sim(dict(base, floating=True))
    for s in (a, b):
        for sp in (0, 1):
            s.load_volume(sp, 20000)
        s.step(1)
    assert np.abs(a.grid("phi") - b.grid("phi")).max() < 1e-12
    for sp in (0, 1):
        pa, pb = a.particles(sp)[0], b.particles(sp)[0]
        assert pa.shape == pb.shape and np.abs(pa - pb).max() < 1e-10
    assert np.allclose(a.history()[0, :10], b.history()[0, :10], rtol=1e-10, atol=1e-12)


def test_grain_charge_is_the_collected_charge():
    """In a plasma the grain charge after n steps is its first charge plus all
    the charge it collected (absorbed and injected-then-absorbed particles),
    and an initially uncharged grain charges negatively (electrons are faster)."""
    cfg = workload(n1=32, n2=16, alpha=0.15, n_init=20000, seed=5, phi_g=0.0, floating=True)
    s = oracle.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, 20000)
    s.step(20)
    h = s.history()
    collected = np.concatenate([[0.0], np.cumsum(h[:-1, 1] * cfg["dt"])])
    scale = np.abs(h[:, 6]).max() + np.abs(collected).max()
    assert np.abs(h[:, 6] - h[0, 6] - collected).max() < 1e-12 * scale
    assert h[-1, 10] < h[0, 10] - 0.05
    assert (np.diff(h[:, 6]) <= 1e-12 * scale).all()  # no step gains positive charge at phi_g ~ 0


def test_floating_needs_a_field():
    with pytest.raises(ValueError):
        oracle.Sim(_vacuum_cfg(32, 16, 0.0, no_field=True))
