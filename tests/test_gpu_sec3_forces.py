"""The simulation example of Sec. 3, at reduced size, checked qualitatively
(the paper shows its forces only as figures): the example's grain (alpha =
-0.24 from Eq. 1 with the printed charge and dipole moment; the grain
potential -2.16 Te/e derived from the printed charge, tests/golden), me/mi =
0.1, Ti = 0.1 Te, Debye length = R0, no magnetic field.  The total force on
the grain along Z (electric, from E_n on the surface, plus the momentum of
the absorbed particles) is clearly nonzero for that grain, while a spherical
grain (alpha = 0) in the same plasma shows none within its noise (Sec. 3's
spherical control run)."""
import numpy as np
import pytest

from tests.inputs import ELECTRON, workload

pytestmark = pytest.mark.gpu


def _force(apic, alpha, n=10_000_000, warm=1500, avg=4000):
    cfg = workload(n1=64, n2=32, alpha=alpha, x1_out=-0.1, phi_g=-2.16, B=0.0, dt=0.1, n_init=n,
                   precision="fp32", sort_interval=8, history_cap=avg + 8, seed=5)
    cfg["species"] = [dict(ELECTRON, n_init=n), dict(q=1.0, m=10.0, T=0.1, n_init=n)]
    s = apic.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, n)
    s.step(warm + avg)
    h = s.tallies()["history"][-avg:]
    s.close()
    f = h[:, 2] + h[:, 3]  # drag F_Z + electric F_Z per step
    means = f.reshape(-1, 50).mean(axis=1)  # means of 50-step batches: their scatter gives the noise
    return f.mean(), means.std(ddof=1) / np.sqrt(len(means))


def test_dipole_grain_feels_a_force_and_the_sphere_none():
    import paper_2307_11107_gb300 as apic
    apic.build()
    f_dip, e_dip = _force(apic, -0.24)
    f_sph, e_sph = _force(apic, 0.0)
    print(f"\nF_Z alpha=-0.24: {f_dip:.4f} +- {e_dip:.4f}; alpha=0: {f_sph:.4f} +- {e_sph:.4f}")
    assert abs(f_sph) < 4.0 * e_sph + 0.01
    assert abs(f_dip) > 5.0 * e_dip
    assert abs(f_dip) > 3.0 * (abs(f_sph) + e_sph)
