"""Boltzmann electrons (APIC_BOLTZMANN): the GPU's Newton solve of
Delta phi = -(rho_i - exp(phi)) and ion-only steps against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from tests.inputs import ION, random_rho

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import torch
    import paper_2307_11107_gb300 as apic
    assert torch.cuda.is_available()
    apic.build()
    return apic


def _cfg(n1=64, n2=32, alpha=0.15, phi_g=-2.5, precision="fp64", **kw):
    d = dict(alpha=alpha, x1_out=-0.1, phi_g=phi_g, phi_out=0.0, B=0.0, dt=0.5, n1=n1, n2=n2,
             species=[dict(ION, n_init=20000)], no_inject=True, boltzmann=True, precision=precision,
             poisson_tol=1e-12, poisson_max_iter=80, newton_iters=12, seed=3)
    d.update(kw)
    return d


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
def test_newton_solve_matches_oracle(apic, alpha, precision):
    """The nonlinear Poisson problem for a given ion density (a positive,
    noisy field around n0 = 1): the GPU's Newton iterations (BiCGSTAB with the
    linear operator's multigrid) reach the oracle's banded-LU Newton solution."""
    cfg = _cfg(alpha=alpha, precision=precision)
    rho = 1.0 + 0.3 * random_rho(64, 32, seed=11)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    g = s.solve_poisson(rho)
    r = o.solve(rho)
    assert np.abs(g - r).max() < 1e-9 * np.abs(r).max()
    assert s.stats()["solver"].startswith("multigrid BiCGSTAB")


def test_single_step_fp64(apic):
    """One FP64 ion-only step from the same volume load (uniform in physical
    volume, so the ion density is n0 up to noise): phi, node gradients, every
    ion and the tallies agree with the oracle."""
    cfg = _cfg(B=0.5)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    s.load_volume(0, 20000)
    o.load_volume(0, 20000)
    s.step(1)
    o.step(1)
    assert o.newton_iterations() > 0
    phi_o = o.grid("phi")
    assert np.abs(s.field("phi") - phi_o).max() < 1e-10 * np.abs(phi_o).max()
    assert np.abs(s.field("G1") - o.grid("G1")).max() < 1e-8 * np.abs(o.grid("G1")).max()
    g, r = s.particles(0), o.particles(0)[0]
    assert g.shape == r.shape
    assert np.abs(g - r).max() < 1e-9
    t = s.tallies(history=True)
    assert abs(t["history"][0, 1] - o.history()[0, 1]) < 1e-12 * abs(o.history()[0, 1])  # ions + electrons
    assert t["counts"][0]["absorbed"] == o.counts()[0]["absorbed"]
    assert t["counts"][0]["escaped"] == o.counts()[0]["escaped"]
    assert np.abs(t["bins"] - o.bins()).max() < 1e-9 * max(np.abs(o.bins()).max(), 1e-300)


def test_ion_only_run_fp32(apic):
    """Twenty FP32 ion-only steps with injection and the default Newton count:
    the solve converges every step and the grain charge follows the oracle's
    (a different random stream in FP32, so within a few per cent)."""
    cfg = _cfg(n1=32, n2=16, precision="fp32", poisson_tol=1e-10, newton_iters=0)
    cfg.pop("no_inject")
    s = apic.Sim(cfg)
    o = oracle.Sim(dict(cfg, precision="fp64"))
    for sim in (s, o):
        sim.load_volume(0, 20000)
        sim.step(20)
    t = s.tallies(history=True)
    hg, ho = t["history"], o.history()
    assert np.isfinite(hg).all()
    assert t["poisson_res"] <= 1e-10
    assert np.abs(hg[:, 6] - ho[:, 6]).max() < 0.03 * np.abs(ho[:, 6]).max()


def test_boltzmann_batch_equals_solo(apic):
    """A Boltzmann instance and a two-species instance in one batch (per-phase
    multigrid kernels, the Newton loop skipping the linear instance) compute
    what each computes alone on the same kernels."""
    import os
    base = dict(alpha=0.1, x1_out=-0.1, phi_g=-2.0, phi_out=0.0, B=0.5, dt=0.2, n1=32, n2=16, seed=4,
                precision="fp64", poisson_tol=1e-12, poisson_max_iter=80)
    from tests.inputs import ELECTRON
    cfgs = [dict(base, species=[dict(ION, n_init=10000)], boltzmann=True, newton_iters=10),
            dict(base, species=[dict(ELECTRON, n_init=10000), dict(ION, n_init=10000)], instance=1)]
    old = os.environ.get("APIC_SOLVER")
    os.environ["APIC_SOLVER"] = "kernels"
    try:
        solo = []
        for c in cfgs:
            s = apic.Sim(c)
            for sp in range(len(c["species"])):
                s.load_volume(sp, 10000)
            s.step(4)
            solo.append((s.field("phi"), s.tallies(history=True)["history"]))
        b = apic.Sim(cfgs)
        for k, c in enumerate(cfgs):
            for sp in range(len(c["species"])):
                b.load_volume(sp, 10000, instance=k)
        b.step(4)
    finally:
        if old is None:
            os.environ.pop("APIC_SOLVER")
        else:
            os.environ["APIC_SOLVER"] = old
    for k in range(2):
        assert np.array_equal(b.field("phi", k), solo[k][0])
        assert np.allclose(b.tallies(k, history=True)["history"], solo[k][1], rtol=1e-12, atol=1e-12)


def test_boltzmann_rejections(apic):
    s = apic.Sim(_cfg())
    with pytest.raises(apic.ApicError, match="BOLTZMANN"):
        s.sensitivity(2)
    with pytest.raises(apic.ApicError):
        apic.Sim(_cfg(floating=True))


def test_boltzmann_electron_current(apic):
    """With no ions, the grain current is the Boltzmann electrons' Maxwellian
    flux alone: -4 pi exp(phi_g) / sqrt(2 pi) for the unit sphere."""
    s = apic.Sim(_cfg(n1=32, n2=16, alpha=0.0, phi_g=-1.5))
    s.step(2)
    h = s.tallies(history=True)["history"]
    assert np.allclose(h[:, 1], -4 * np.pi * np.exp(-1.5) / np.sqrt(2 * np.pi), rtol=1e-12, atol=0)
