"""Pins of the oracle's field gather (Eq. 10 and the sentence after it), the
electric half-kicks of the Boris push (Eq. 9) and the grain's surface charge
and electric force (Sec. 2, after Eq. 10).

Each check compares the oracle with quantities computed here without it:
gradients of Eq. 2 taken by complex-step differentiation of x1(R, Z) and
x2(R, Z) (exact to rounding), the grain surface as the curve x1 = -1 of Eq. 2
with its area element 2 pi R |dP/dx2| taken from that curve (not from Eq. 4),
and adaptive quadrature of the surface integrals.  The potentials are set
directly on the nodes (oracle.Sim.set_phi), so the node gradients are exact:
linear potentials have exact central and one-sided second-order differences,
and the surface potential below is quadratic in x1.
"""
import numpy as np
import pytest

import oracle

EL = dict(q=-1.0, m=1.0, T=1.0)
ION = dict(q=1.0, m=1836.0, T=1.0)


def _x1(alpha, R, Z):
    """Eq. 2 in cylindrical coordinates (complex-safe)."""
    r = np.sqrt(R * R + Z * Z)
    return -(1.0 / r) * (1.0 + alpha * Z / (r * r))


def _x2(alpha, R, Z):
    return Z / np.sqrt(R * R + Z * Z)


def _grad(f, alpha, R, Z, h=1e-30):
    """(df/dR, df/dZ) by complex-step differentiation."""
    return np.array([f(alpha, R + 1j * h, Z).imag / h, f(alpha, R, Z + 1j * h).imag / h])


def _nodes(n1, n2, x1_out):
    x1 = -1.0 + np.arange(n1 + 1) * ((x1_out + 1.0) / n1)
    x1[-1] = x1_out
    x2 = -1.0 + np.arange(n2 + 1) * (2.0 / n2)
    x2[-1] = 1.0
    return np.meshgrid(x1, x2, indexing="ij")


def _state(alpha, R, Z, vR, vZ, vT):
    return np.array([[_x1(alpha, R, Z), _x2(alpha, R, Z), vR, vZ, vT]])


def _sim(alpha, species, n1=40, n2=24, x1_out=-0.05, dt=0.1, B=0.0):
    d = dict(alpha=alpha, x1_out=x1_out, phi_g=0.0, phi_out=0.0, B=B, dt=dt, n1=n1, n2=n2,
             species=[dict(species, n_init=1000)], no_inject=True)
    return oracle.Sim(d)


def _set_linear_phi(s, n1, n2, x1_out, a, c, d0=0.7):
    X1, X2 = _nodes(n1, n2, x1_out)
    s.set_phi(d0 + a * X1 + c * X2)
    s.gradients()


# (alpha, R, Z) points spread over the domain, away from the grain and the axis
POINTS = [(0.0, 3.0, 0.5), (0.15, 1.6, -1.1), (0.15, 0.4, 2.5), (-0.24, 2.2, 1.9), (0.225, 5.0, -4.0)]


# quadratic potential phi = d + a x1 + c x2 + (a2 x1^2 + c2 x2^2) / 2 + e x1 x2
QUAD = dict(d=0.7, a=1.7, c=-0.9, a2=2.3, c2=-1.1, e=0.8)


def _phi_quad(x1, x2, k=QUAD):
    return k["d"] + k["a"] * x1 + k["c"] * x2 + 0.5 * (k["a2"] * x1 * x1 + k["c2"] * x2 * x2) + k["e"] * x1 * x2


@pytest.mark.parametrize("alpha,R,Z", POINTS)
@pytest.mark.parametrize("sp", [EL, ION])
def test_kick_from_rest_in_quadratic_potential(alpha, R, Z, sp):
    """A potential quadratic in (x1, x2) has exact node gradients (central and
    one-sided second-order differences are exact on quadratics), and they are
    linear in (x1, x2), so the bilinear gather reproduces them exactly at the
    particle: the gathered field is E = -(dphi/dx1 grad x1 + dphi/dx2 grad x2)
    there (Eq. 10).  A particle at rest with B = 0 leaves its first step with
    v = (q/m) dt E (the two electric half-kicks of Eq. 9) and moves by v dt.
    A flipped sign of E, a swapped metric entry or interpolation weight, or a
    lost half-kick fails this."""
    n1, n2, x1_out, dt = 40, 24, -0.05, 0.1
    k = QUAD
    s = _sim(alpha, sp, n1, n2, x1_out, dt)
    X1, X2 = _nodes(n1, n2, x1_out)
    s.set_phi(_phi_quad(X1, X2))
    s.gradients()
    s.add_particles(0, _state(alpha, R, Z, 0.0, 0.0, 0.0))
    s.push_only()
    st, _ = s.particles(0)
    assert st.shape[0] == 1
    x1, x2 = _x1(alpha, R, Z), _x2(alpha, R, Z)
    d1 = k["a"] + k["a2"] * x1 + k["e"] * x2
    d2 = k["c"] + k["c2"] * x2 + k["e"] * x1
    E = -(d1 * _grad(_x1, alpha, R, Z) + d2 * _grad(_x2, alpha, R, Z))
    v = sp["q"] / sp["m"] * dt * E
    scale = np.abs(v).max()
    assert abs(st[0, 2] - v[0]) <= 1e-12 * scale
    assert abs(st[0, 3] - v[1]) <= 1e-12 * scale
    assert abs(st[0, 4]) <= 1e-15 * scale
    # the new position: the start plus v dt, back in (x1, x2)
    Rn, Zn = R + v[0] * dt, Z + v[1] * dt
    assert st[0, 0] == pytest.approx(_x1(alpha, Rn, Zn), rel=1e-13, abs=1e-15)
    assert st[0, 1] == pytest.approx(_x2(alpha, Rn, Zn), rel=1e-13, abs=1e-15)


def _energy_drift(alpha, a, c, dt, t_end, start, sp=EL, B=0.0):
    """Largest |W - W_0| along an orbit in the static potential
    phi = a x1 + c x2, W = m |v^{n+1/2}|^2 / 2 + q (phi(x^n) + phi(x^{n+1})) / 2
    (kinetic energy at the half step, potential energy time-centred)."""
    n1, n2, x1_out = 64, 32, -0.05
    s = _sim(alpha, sp, n1, n2, x1_out, dt, B=B)
    _set_linear_phi(s, n1, n2, x1_out, a, c, d0=0.0)
    R, Z, vR, vZ, vT = start
    st = _state(alpha, R, Z, vR, vZ, vT)
    s.add_particles(0, st)
    q, m = sp["q"], sp["m"]

    def phi(row):
        return a * row[0] + c * row[1]

    W = []
    prev = st[0]
    for _ in range(int(round(t_end / dt))):
        s.push_only()
        cur, _ = s.particles(0)
        assert cur.shape[0] == 1, "the orbit left the domain"
        cur = cur[0]
        W.append(0.5 * m * (cur[2:] ** 2).sum() + q * 0.5 * (phi(prev) + phi(cur)))
        prev = cur
    W = np.array(W)
    return np.abs(W - W[0]).max(), np.abs(W).max()


@pytest.mark.parametrize("alpha,c,B,start", [
    (0.0, 0.0, 0.0, (3.0, 0.0, 0.1, 0.55, 0.35)),
    (0.15, 0.2, 0.0, (4.0, 0.0, 0.0, 0.45, 0.4)),
    (0.15, 0.1, 0.3, (3.0, 1.0, 0.0, 0.5, 0.4)),
    (-0.24, -0.15, 0.4, (3.0, 1.0, 0.0, 0.5, 0.4))])
def test_energy_conserved_in_static_potential(alpha, c, B, start):
    """In a static potential the time-centred leapfrog conserves
    kinetic + potential energy up to an O(dt^2) oscillation (the magnetic
    rotation does no work).  With alpha = 0 and c = 0, phi = a x1 = -a/r is a
    Coulomb potential and the electron moves on a Kepler ellipse.  A wrong
    sign or magnitude of the electric kick gives an O(1) energy error."""
    a = -2.0  # start: R, Z, vR, vZ, vT of a bound orbit that stays inside the domain
    e1, w = _energy_drift(alpha, a, c, 0.1, 60.0, start, B=B)
    e2, _ = _energy_drift(alpha, a, c, 0.05, 60.0, start, B=B)
    assert e1 < 1e-2 * w
    assert 3.5 < e1 / e2 < 4.5


def _surface_exact(alpha, g):
    """Q = int E_n dA and F_Z = int (E_n^2 / 2) n_Z dA over the grain x1 = -1
    for a potential whose normal derivative there is dphi/dx1 = g(x2):
    E_n = -g |grad x1|, n_Z = (dx1/dZ) / |grad x1|, the surface the curve
    P(x2) = r_g(x2) (sqrt(1 - x2^2), x2) with r_g from Eq. 2 at x1 = -1
    (r^2 = r + alpha x2), dA = 2 pi R |dP/dx2| dx2."""
    from scipy.integrate import quad

    def curve(x2):
        rg = (1.0 + np.sqrt(1.0 + 4.0 * alpha * x2)) / 2.0
        return rg * np.sqrt((1.0 - x2) * (1.0 + x2)), rg * x2

    def parts(x2):
        h = 1e-30
        Rc, Zc = curve(x2)
        dR, dZ = (np.array(curve(x2 + 1j * h)) .imag / h)
        gx = _grad(_x1, alpha, Rc, Zc)
        gn = np.hypot(*gx)
        En = -g(x2) * gn
        dA = 2.0 * np.pi * Rc * np.hypot(dR, dZ)
        return En, gx[1] / gn, dA

    Q = quad(lambda x: parts(x)[0] * parts(x)[2], -1.0, 1.0, epsabs=0, epsrel=1e-13, limit=200)[0]
    FZ = quad(lambda x: 0.5 * parts(x)[0] ** 2 * parts(x)[1] * parts(x)[2], -1.0, 1.0, epsabs=0,
              epsrel=1e-13, limit=200)[0]
    return Q, FZ


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_surface_charge_and_force_against_surface_integrals(alpha):
    """phi = phi_g + (x1 + 1)(1 + 0.3 (x1 + 1)) g(x2), g = 3 + x2 + x2^2 / 2:
    constant on the grain, quadratic in x1 (so the one-sided second-order
    dphi/dx1 on the grain is exact), with a normal field that differs between
    the two ends of the grain, so F_Z != 0.  The oracle's trapezoid sums of
    Q and F_Z converge to the surface integrals at second order in h2.  A
    lost factor 1/2, a wrong normal component, area element or sign fails."""
    n1, x1_out, pg = 24, -0.1, -2.5

    def g(x2):
        return 3.0 + x2 + 0.5 * x2 * x2

    Qx, Fx = _surface_exact(alpha, g)
    assert abs(Fx) > 0.05 * abs(Qx)  # the force is not small against the charge
    errs = []
    for n2 in (32, 64, 128):
        s = _sim(alpha, EL, n1, n2, x1_out)
        X1, X2 = _nodes(n1, n2, x1_out)
        s.set_phi(pg + (X1 + 1.0) * (1.0 + 0.3 * (X1 + 1.0)) * g(X2))
        s.gradients()
        En, Q, FZ = s.surface()
        errs.append((abs(Q - Qx) / abs(Qx), abs(FZ - Fx) / abs(Fx)))
    errs = np.array(errs)
    assert errs[-1].max() < 1e-3, errs
    rates = np.log2(errs[:-1] / errs[1:])
    assert (rates > 1.8).all(), (errs, rates)
