"""Pins of the oracle's particle mover (Eq. 9, Sec. 2 leapfrog), absorption,
escape and injection (Sec. 1), and of the whole step's bookkeeping."""
import numpy as np
import pytest

import oracle

EL = dict(q=-1.0, m=1.0, T=1.0)


def _free_cfg(**kw):
    d = dict(alpha=0.0, x1_out=-0.05, phi_g=0.0, phi_out=0.0, B=0.0, dt=0.1, n1=16, n2=8,
             species=[dict(EL, n_init=1000)], no_field=True, no_inject=True)
    d.update(kw)
    return d


def _state_at(alpha, R, Z, vR, vZ, vT):
    r = np.hypot(R, Z)
    x2 = Z / r
    return np.array([[oracle.x1_of(alpha, r, x2), x2, vR, vZ, vT]])


def _RZ(alpha, st):
    x1, x2 = st[0, 0], st[0, 1]
    r = oracle.r_of(alpha, x1, x2)
    return r * np.sqrt((1 - x2) * (1 + x2)), r * x2


@pytest.mark.parametrize("alpha", [0.0, 0.2])
def test_free_streaming_is_a_straight_line(alpha):
    """E = 0, B = 0: the cylindrical mover (chord + rotation back to the
    meridional plane, which carries the V_Theta^2/R and -V_R V_Theta/R terms of
    Eq. 9) moves on the exact Cartesian straight line."""
    R0, Z0, v = 6.0, -2.0, np.array([0.3, 0.2, 0.7])  # (vR, vZ, vT)
    s = oracle.Sim(_free_cfg(alpha=alpha))
    s.add_particles(0, _state_at(alpha, R0, Z0, *v))
    for k in range(1, 41):
        s.push_only()
        st, _ = s.particles(0)
        t = 0.1 * k
        x, y, z = R0 + v[0] * t, v[2] * t, Z0 + v[1] * t
        R = np.hypot(x, y)
        Rn, Zn = _RZ(alpha, st)
        assert Rn == pytest.approx(R, rel=1e-12) and Zn == pytest.approx(z, rel=1e-12, abs=1e-12)
        vR, vT = (x * v[0] + y * v[2]) / R, (-y * v[0] + x * v[2]) / R
        assert st[0, 2] == pytest.approx(vR, rel=1e-11, abs=1e-12)
        assert st[0, 4] == pytest.approx(vT, rel=1e-11, abs=1e-12)
        assert st[0, 3] == pytest.approx(v[1], rel=1e-14)


def _gyro_error(n_per_period, q=-1.0, m=1.0, B=1.0):
    """Position error after one gyro period 2 pi m / (|q| B), pure B."""
    T = 2 * np.pi * m / (abs(q) * B)
    dt = T / n_per_period
    s = oracle.Sim(_free_cfg(B=B, dt=dt, species=[dict(q=q, m=m, T=1.0, n_init=1000)]))
    st0 = _state_at(0.0, 5.0, 0.5, 0.3, 0.05, 0.4)
    s.add_particles(0, st0)
    speeds = []
    for _ in range(n_per_period):
        s.push_only()
        st, _ = s.particles(0)
        speeds.append(np.linalg.norm(st[0, 2:]))
    R0, Z0 = _RZ(0.0, st0)
    R1, Z1 = _RZ(0.0, st)
    vz_drift = 0.05 * T
    return np.hypot(R1 - R0, Z1 - (Z0 + vz_drift)), np.array(speeds), st


def test_gyro_orbit_closes_second_order():
    """Pure B along the axis: the orbit closes after one period 2 pi m/(|q| B)
    with an O(dt^2) phase error (time-centred leapfrog), and |v| is conserved to
    rounding (magnetic rotation)."""
    e64, sp64, _ = _gyro_error(64)
    e128, sp128, _ = _gyro_error(128)
    assert e64 < 5e-3
    assert 3.3 < e64 / e128 < 4.7
    v0 = np.linalg.norm([0.3, 0.05, 0.4])
    assert np.abs(sp64 - v0).max() < 1e-13
    assert np.abs(sp128 - v0).max() < 1e-13


def test_canonical_angular_momentum_exact():
    """From Eq. 9, d(R V_Theta)/dt = (q/m) B R V_R, so R V_Theta - (q/m) B R^2/2
    is conserved (E_Theta = 0).  With the velocity at n+1/2 and R^2 taken at the
    chord midpoint (time-centred), the discrete mover conserves it to rounding."""
    for n in (32, 96):
        dt = 2 * np.pi / n
        s = oracle.Sim(_free_cfg(B=1.0, dt=dt))
        s.add_particles(0, _state_at(0.0, 4.0, 0.0, 0.2, 0.0, 0.5))
        qm, vals = -1.0, []
        for _ in range(3 * n):
            s.push_only()
            st, _ = s.particles(0)
            R, _ = _RZ(0.0, st)
            vR, vT = st[0, 2], st[0, 4]
            Rmid2 = (R - vR * dt / 2) ** 2 + (vT * dt / 2) ** 2
            vals.append(R * vT - qm * 1.0 * Rmid2 / 2)
        vals = np.array(vals)
        assert np.abs(vals - vals[0]).max() < 1e-13 * abs(vals[0])


def test_radial_infall_impact_point_and_tallies():
    """A particle moving straight at the sphere along a ray is absorbed at the
    polar angle of that ray; the tally carries its charge, momentum and energy
    (Sec. 1: transferred locally at the point of impact)."""
    alpha = 0.0
    cfg = _free_cfg(alpha=alpha, dt=0.5, n2=16)
    s = oracle.Sim(cfg)
    x2 = 0.3
    r0 = 1.2
    u = np.array([np.sqrt(1 - x2 * x2), x2])  # (R, Z) direction of the ray
    vel = -0.9 * u
    st = _state_at(alpha, r0 * u[0], r0 * u[1], vel[0], vel[1], 0.0)
    s.add_particles(0, st)
    s.push_only()
    assert s.count(0) == 0
    bins = s.bins()[0]
    k = int(np.floor((x2 + 1) / (2 / 16)))
    assert bins[k, 0] == 1.0 and bins.sum(axis=0)[0] == 1.0
    w = s.scalars()["w0"]
    assert bins[k, 1] == pytest.approx(-1.0 * w)
    assert bins[k, 2] == pytest.approx(vel[0] * w, rel=1e-12)  # radial (R) momentum at impact azimuth
    assert bins[k, 3] == pytest.approx(vel[1] * w, rel=1e-12)
    assert bins[k, 4] == pytest.approx(0.0, abs=1e-15)
    assert bins[k, 5] == pytest.approx(0.5 * 0.81 * w, rel=1e-12)


def test_binding_energy_counts_for_positive_charges_only():
    """The heat-flux component of the tallies (E_kin + E_bind) adds the
    binding energy per absorbed particle of positive charge (weighted like
    every tally), and nothing for electrons (Sec. 1: energy transferred to
    the grain at the point of impact)."""
    e_bind = 3.5
    cfg = _free_cfg(dt=0.5, n2=16, e_bind_ion=e_bind,
                    species=[dict(EL, n_init=1000), dict(q=1.0, m=1836.0, T=1.0, n_init=1000)])
    s = oracle.Sim(cfg)
    for sp, x2, speed in ((0, 0.3, 0.9), (1, -0.4, 0.7)):
        u = np.array([np.sqrt(1 - x2 * x2), x2])
        st = _state_at(0.0, 1.2 * u[0], 1.2 * u[1], -speed * u[0], -speed * u[1], 0.0)
        s.add_particles(sp, st)
    s.push_only()
    assert s.count(0) == 0 and s.count(1) == 0
    b = s.bins()
    sc = s.scalars()
    for sp, m, speed, w in ((0, 1.0, 0.9, sc["w0"]), (1, 1836.0, 0.7, sc["w1"])):
        hit = b[sp][:, 0] > 0
        assert hit.sum() == 1
        ek = b[sp][hit, 5][0]
        assert ek == pytest.approx(0.5 * m * speed * speed * w, rel=1e-12)
        extra = b[sp][hit, 6][0] - ek
        assert extra == pytest.approx(e_bind * w if sp == 1 else 0.0, rel=1e-12, abs=1e-300)


@pytest.mark.slow
def test_field_free_thermal_flux_to_sphere():
    """No field: the absorption rate onto a convex grain in a uniform isotropic
    Maxwellian is n0 sqrt(T / 2 pi m) A_grain, A_grain = 4 pi for a sphere."""
    n_init = 20000
    cfg = _free_cfg(alpha=0.0, x1_out=-0.1, dt=0.1, n1=16, n2=8,
                    species=[dict(EL, n_init=n_init)], no_inject=False)
    s = oracle.Sim(cfg)
    s.load_volume(0, n_init)
    steps = 400
    s.step(steps)
    c = s.counts()[0]
    w = s.scalars()["w0"]
    expect = np.sqrt(1.0 / (2 * np.pi)) * 4 * np.pi * 0.1 * steps / w
    assert abs(c["absorbed"] - expect) < 4.5 * np.sqrt(expect)
    assert c["loaded"] + c["injected"] == c["absorbed"] + c["escaped"] + c["resident"]


@pytest.mark.slow
@pytest.mark.parametrize("alpha", [0.0, 0.15])
def test_injection_fills_empty_domain_to_n0(alpha):
    """Surface injection alone (Sec. 1, Eq. 4 at x1_out) with the flux-weighted
    half-Maxwellian fills an empty domain to density n0 (the particle count
    tends to V_domain / w, less the small shadow of the absorbing grain)."""
    n_init = 10000
    cfg = _free_cfg(alpha=alpha, x1_out=-0.1, dt=0.1, n1=16, n2=8,
                    species=[dict(EL, n_init=n_init)], no_inject=False)
    s = oracle.Sim(cfg)
    s.step(400)
    res = s.counts()[0]["resident"]
    hist = s.history()
    avg = hist[-100:, 7].mean()
    assert 0.95 * n_init < avg < 1.0 * n_init, (avg, res)
    c = s.counts()[0]
    assert c["loaded"] + c["injected"] == c["absorbed"] + c["escaped"] + c["resident"]


def test_count_balance_and_history_with_field():
    """A short self-consistent run: integer count balance per species, history
    rows for every step, finite diagnostics."""
    cfg = dict(alpha=0.15, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, B=0.5, dt=0.1, n1=32, n2=16,
               species=[dict(EL, n_init=20000), dict(q=1.0, m=1836.0, T=1.0, n_init=20000)], seed=3)
    s = oracle.Sim(cfg)
    s.load_volume(0, 20000)
    s.load_volume(1, 20000)
    s.step(20)
    for c in s.counts():
        assert c["loaded"] + c["injected"] == c["absorbed"] + c["escaped"] + c["resident"]
    h = s.history()
    assert h.shape == (20, 11) and np.isfinite(h).all()
    b = s.bins()
    assert b[:, :, 0].sum() == sum(c["absorbed"] for c in s.counts())


@pytest.mark.parametrize("alpha", [0.0, 0.2])
def test_deposit_uniform_load_gives_n0(alpha):
    """Charge weighing with the hat-weighted node volumes (Eq. 5): a load that
    is uniform in physical volume gives rho = n0 in expectation at every node
    (checked per x1 row against its Poisson error), and the total charge
    sum(rho V) equals q w N exactly (CIC weights sum to one)."""
    n = 200000
    cfg = dict(alpha=alpha, x1_out=-0.3, phi_g=0, phi_out=0, B=0, dt=0.1, n1=16, n2=8,
               species=[dict(q=1.0, m=1.0, T=1.0, n_init=n)], no_field=True, no_inject=True)
    s = oracle.Sim(cfg)
    s.load_volume(0, n)
    s.deposit()
    rho, V = s.grid("rho"), s.grid("V")
    w = s.scalars()["w0"]
    assert (rho * V).sum() == pytest.approx(w * n, rel=1e-12)
    for i in range(rho.shape[0]):
        Vi = V[i].sum()
        mean = (rho[i] * V[i]).sum() / Vi
        sigma = np.sqrt(w / Vi)  # Poisson bound: sum of CIC weights^2 <= sum of weights
        assert abs(mean - 1.0) < 5 * sigma, (i, mean, sigma)


def test_chord_option_absorbs_grazing_orbits():
    """A fast particle whose straight chord crosses the spherical grain but
    ends outside it: without the option the end-point test lets it through;
    with the chord option it is absorbed where the chord enters the grain
    (impact point on the sphere, bin of that polar angle)."""
    dt = 1.0
    for chord in (False, True):
        cfg = _free_cfg(dt=dt, n2=16, chord_absorb=chord)
        s = oracle.Sim(cfg)
        # from (R, Z) = (0.5, -1.5) straight up at 3 per unit time: the chord
        # enters the unit sphere at Z = -sqrt(0.75) and ends at Z = 1.5
        st = _state_at(0.0, 0.5, -1.5, 0.0, 3.0, 0.0)
        s.add_particles(0, st)
        s.push_only()
        if not chord:
            assert s.count(0) == 1
            continue
        assert s.count(0) == 0
        b = s.bins()[0]
        k = int(np.floor((-np.sqrt(0.75) + 1) / (2 / 16)))
        assert b[k, 0] == 1.0 and b[:, 0].sum() == 1.0


def test_chord_option_keeps_chords_that_miss():
    """A chord that passes outside the grain is not absorbed with the option,
    and the particle moves exactly as without it."""
    runs = []
    for chord in (False, True):
        cfg = _free_cfg(dt=1.0, n2=16, chord_absorb=chord)
        s = oracle.Sim(cfg)
        s.add_particles(0, _state_at(0.0, 1.3, -1.5, 0.0, 3.0, 0.0))
        s.push_only()
        assert s.count(0) == 1
        runs.append(s.particles(0)[0])
    assert np.array_equal(runs[0], runs[1])
