"""Isolated grain (APIC_FLOATING): the GPU path against the closed form of a
charged sphere in its grounded shell and against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests.inputs import ELECTRON, ION, random_states, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import torch
    import paper_2307_11107_gb300 as apic
    assert torch.cuda.is_available()
    apic.build()
    return apic


def _vacuum_cfg(phi_g, precision, **kw):
    d = dict(alpha=0.0, x1_out=-0.1, phi_g=phi_g, phi_out=0.0, B=0.0, dt=0.1, n1=64, n2=32,
             species=[dict(ELECTRON, n_init=10000), dict(ION, n_init=10000)], no_inject=True,
             floating=True, precision=precision, poisson_tol=1e-12, poisson_max_iter=60)
    d.update(kw)
    return d


def _shell_capacitance(x1_out):
    """4 pi / (1/r_g - 1/r_out): unit sphere in a concentric grounded shell."""
    return 4 * np.pi / (1.0 - 1.0 / oracle.r_of(0.0, x1_out, 0.3))


def _ions_falling_in(n, r0, v0, seed):
    rng = np.random.default_rng(seed)
    x2 = rng.uniform(-0.95, 0.95, n)
    R, Z = r0 * np.sqrt(1 - x2 * x2), r0 * x2
    x1 = np.array([oracle.x1_of(0.0, r0, c) for c in x2])
    return np.column_stack([x1, x2, -v0 * R / r0, -v0 * Z / r0, np.zeros(n)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_charged_sphere_in_its_shell(apic, precision):
    """Vacuum: the first step's grain charge is C phi_g (C of the shell: the
    vacuum field is linear in x1 = -1/r, so exact on the grid); ions falling
    onto the grain leave its charge unchanged while they approach and, once
    absorbed, raise its potential by N q w / C."""
    phi_g = -1.0
    s = apic.Sim(_vacuum_cfg(phi_g, precision))
    s.step(1)
    C = _shell_capacitance(-0.1)
    tol = 1e-9
    h = s.tallies(history=True)["history"]
    Q0 = h[0, 6]
    assert Q0 == pytest.approx(C * phi_g, rel=tol)
    assert h[0, 10] == phi_g
    n = 300
    s.add_particles(1, _ions_falling_in(n, 1.05, 2.0, seed=4))
    s.step(2)
    t = s.tallies(history=True)
    h = t["history"]
    assert t["counts"][1]["absorbed"] == n
    w = oracle.Sim(_vacuum_cfg(phi_g, "fp64")).scalars()["w1"]
    dq = n * w
    assert h[1, 6] == pytest.approx(Q0, rel=tol)
    assert abs(h[1, 10] - phi_g) > 1e-4
    assert h[2, 6] == pytest.approx(Q0 + dq, rel=tol)
    assert h[2, 10] - phi_g == pytest.approx(dq / C, rel=1e-8 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("alpha,B", [(0.15, 0.5), (-0.24, 1.0)])
def test_floating_steps_fp64_match_oracle(apic, alpha, B):
    """Four FP64 steps of an isolated grain from identical explicit states:
    grain charge and potential histories, phi, the particles and the counts
    agree with the oracle."""
    cfg = workload(n1=64, n2=32, alpha=alpha, B=B, n_init=20000, precision="fp64", no_inject=True,
                   phi_g=-0.5, poisson_tol=1e-13, poisson_max_iter=60, floating=True)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp, seed, vs in ((0, 21, 1.0), (1, 22, 0.03)):
        st = random_states(20000, cfg["x1_out"], seed=seed, vscale=vs)
        s.add_particles(sp, st)
        o.add_particles(sp, st)
    s.step(4)
    o.step(4)
    hg, ho = s.tallies(history=True)["history"], o.history()
    assert hg.shape == ho.shape == (4, 11)
    assert np.abs(hg[:, 10] - ho[:, 10]).max() < 1e-9
    assert np.abs(hg[:, 6] - ho[:, 6]).max() < 1e-9 * np.abs(ho[:, 6]).max()
    assert np.abs(hg[:, 3] - ho[:, 3]).max() < 1e-8 * np.abs(ho[:, 3]).max()
    assert abs(ho[-1, 10] - ho[0, 10]) > 1e-3  # the potential did move
    phi_o = o.grid("phi")
    assert np.abs(s.field("phi") - phi_o).max() < 1e-10 * np.abs(phi_o).max()
    for sp in (0, 1):
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape
        assert np.abs(g - r).max() < 1e-8
        assert s.tallies()["counts"][sp]["absorbed"] == o.counts()[sp]["absorbed"]


def test_floating_fp32_tracks_oracle(apic):
    """FP32 particles with the refined solve: 20 steps with injection; the
    grain potential stays within its statistical noise of the FP64 oracle's
    (both charge the grain negatively from 0)."""
    cfg = workload(n1=32, n2=16, alpha=0.15, n_init=40000, seed=5, phi_g=0.0, floating=True)
    s = apic.Sim(dict(cfg, precision="fp32"))
    o = oracle.Sim(dict(cfg, precision="fp64"))
    for sim in (s, o):
        for sp in (0, 1):
            sim.load_volume(sp, 40000)
        sim.step(20)
    hg, ho = s.tallies(history=True)["history"], o.history()
    assert hg[-1, 10] < -0.1 and ho[-1, 10] < -0.1
    collected = np.concatenate([[0.0], np.cumsum(hg[:-1, 1] * cfg["dt"])])
    assert np.abs(hg[:, 6] - hg[0, 6] - collected).max() < 1e-9 * np.abs(hg[:, 6]).max()
    assert abs(hg[-1, 10] - ho[-1, 10]) < 0.5 * abs(ho[-1, 10])  # seeds spread by ~20 %


def test_floating_batch_equals_solo(apic):
    """An isolated grain and a fixed-potential grain in one batch (one batched
    reduction solve) compute what each computes alone."""
    base = workload(n1=32, n2=16, alpha=0.1, n_init=10000, seed=7, phi_g=-0.3, precision="fp32")
    cfgs = [dict(base, floating=True), dict(base, instance=1)]
    solo = []
    for c in cfgs:
        s = apic.Sim(c)
        for sp in (0, 1):
            s.load_volume(sp, 10000)
        s.step(5)
        solo.append((s.tallies(history=True)["history"], s.field("phi")))
    b = apic.Sim(cfgs)
    for k in range(2):
        for sp in (0, 1):
            b.load_volume(sp, 10000, instance=k)
    b.step(5)
    for k in range(2):
        hb = b.tallies(history=True, instance=k)["history"]
        assert np.allclose(hb, solo[k][0], rtol=1e-12, atol=1e-12)
        assert np.array_equal(b.field("phi", k), solo[k][1])
    assert solo[0][0][-1, 10] != solo[0][0][0, 10]


def test_floating_rejected_by_sensitivity(apic):
    s = apic.Sim(_vacuum_cfg(-1.0, "fp64"))
    with pytest.raises(apic.ApicError, match="FLOATING"):
        s.sensitivity(2)


def test_floating_needs_a_field(apic):
    with pytest.raises(apic.ApicError):
        apic.Sim(_vacuum_cfg(-1.0, "fp64", no_field=True))
