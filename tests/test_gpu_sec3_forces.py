"""The simulation example of Sec. 3, at reduced size, checked qualitatively
(the paper shows its forces only as figures): the example's grain (alpha =
-0.24 from Eq. 1 with the printed charge and dipole moment; the grain
potential -2.16 Te/e derived from the printed charge, tests/golden), me/mi =
0.1, Ti = 0.1 Te, Debye length = R0, no magnetic field.  The total force on
the grain along Z (electric, from E_n on the surface, plus the momentum of
the absorbed particles) is clearly nonzero for that grain, while a spherical
grain (alpha = 0) in the same plasma shows none within its noise (Sec. 3's
spherical control run).

The same runs check Sec. 3's screening features: at equal x1 the potential
is more positive near the 'dull' end x2 = +1 than near the 'sharp' end
x2 = -1 (in vacuum it depends on x1 alone, Eq. 7 having no first x1
derivative), and positive charge gathers near the ends of the grain; the
sphere shows neither asymmetry."""
import numpy as np
import pytest

from tests.inputs import ELECTRON, workload

pytestmark = pytest.mark.gpu


def _run(apic, alpha, n=10_000_000, warm=1500, avg=4000, every=20):
    cfg = workload(n1=64, n2=32, alpha=alpha, x1_out=-0.1, phi_g=-2.16, B=0.0, dt=0.1, n_init=n,
                   precision="fp32", sort_interval=8, history_cap=avg + 8, seed=5)
    cfg["species"] = [dict(ELECTRON, n_init=n), dict(q=1.0, m=10.0, T=0.1, n_init=n)]
    s = apic.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, n)
    s.step(warm)
    phi, rho = [], []
    for _ in range(avg // every):
        s.step(every)
        phi.append(s.field("phi"))
        rho.append(s.field("rho"))
    h = s.tallies()["history"][-avg:]
    s.close()
    f = h[:, 2] + h[:, 3]  # drag F_Z + electric F_Z per step
    means = f.reshape(-1, 50).mean(axis=1)  # means of 50-step batches: their scatter gives the noise
    return dict(force=(f.mean(), means.std(ddof=1) / np.sqrt(len(means))), phi=np.array(phi), rho=np.array(rho))


def _batch_stat(samples, nb=10):
    """Mean and standard error of a per-sample statistic from nb batch means."""
    b = samples.reshape(nb, -1, *samples.shape[1:]).mean(axis=1)
    return b.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(nb)


@pytest.fixture(scope="module")
def runs():
    import paper_2307_11107_gb300 as apic
    apic.build()
    return {a: _run(apic, a) for a in (-0.24, 0.0)}


def test_dipole_grain_feels_a_force_and_the_sphere_none(runs):
    f_dip, e_dip = runs[-0.24]["force"]
    f_sph, e_sph = runs[0.0]["force"]
    print(f"\nF_Z alpha=-0.24: {f_dip:.4f} +- {e_dip:.4f}; alpha=0: {f_sph:.4f} +- {e_sph:.4f}")
    assert abs(f_sph) < 4.0 * e_sph + 0.01
    assert abs(f_dip) > 5.0 * e_dip
    assert abs(f_dip) > 3.0 * (abs(f_sph) + e_sph)


def test_screening_asymmetry_of_the_potential(runs):
    """phi near x2 = +1 minus phi near x2 = -1 (three nodes at each end), rows
    2-8 next to the grain: clearly positive for the dipole grain, zero within
    noise for the sphere."""
    for alpha in (-0.24, 0.0):
        P = runs[alpha]["phi"]
        m, e = _batch_stat(P[:, :, -3:].mean(axis=2) - P[:, :, :3].mean(axis=2))
        print(f"\nalpha={alpha}: dphi rows 2, 4, 8 = {m[2]:+.5f} +- {e[2]:.5f}, {m[4]:+.5f} +- {e[4]:.5f}, "
              f"{m[8]:+.5f} +- {e[8]:.5f}")
        for i in (2, 4, 8):
            if alpha == 0.0:
                assert abs(m[i]) < 4.0 * e[i] + 1e-4
            else:
                assert m[i] > 10.0 * e[i] and m[i] > 0.002


def test_positive_charge_gathers_at_the_grain_ends(runs):
    """The charge density on the first row off the dipole grain is larger at
    its ends (three nodes at each of x2 = +-1) than around its middle."""
    R = runs[-0.24]["rho"][:, 1, :]
    ends = 0.5 * (R[:, -3:].mean(axis=1) + R[:, :3].mean(axis=1))
    mid = R[:, 14:19].mean(axis=1)
    m, e = _batch_stat(ends - mid)
    print(f"\nrho ends - middle (row 1, alpha=-0.24): {m:+.4f} +- {e:.4f}")
    assert m > 2.0 * e and m > 0.0
