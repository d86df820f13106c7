"""Conservative operator (APIC_FE_OPERATOR): the GPU's solvers on the bilinear
finite-element form of Eqs. 6-7 against the oracle's banded LU of the same
form, and one full step."""
import numpy as np
import pytest

import oracle
from tests.inputs import random_rho, random_states, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import torch
    import paper_2307_11107_gb300 as apic
    assert torch.cuda.is_available()
    apic.build()
    return apic


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("alpha", [0.0, 0.15, -0.24])
@pytest.mark.parametrize("precision,grid", [("fp64", (64, 32)), ("fp64", (96, 48)), ("fp32", (128, 64)),
                                            ("fp32", (160, 80))])
def test_poisson_matches_banded_lu(apic, alpha, precision, grid):
    """The multigrid BiCGSTAB (FP64 form) and the block cyclic reduction in
    FP64 refinement (FP32 form) solve the conservative system to the
    oracle's LU solution."""
    n1, n2 = grid
    cfg = workload(n1=n1, n2=n2, alpha=alpha, n_init=1000, precision=precision, fe_operator=True,
                   poisson_tol=1e-12, poisson_max_iter=80)
    rho = random_rho(n1, n2, seed=n1 + 7, scale=0.3)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    if precision == "fp32":
        assert s.stats()["solver"].startswith("FP32 block cyclic reduction")
    assert rel(s.solve_poisson(rho), o.solve(rho)) < 1e-9


def test_single_step_fp64(apic):
    """One FP64 step with the conservative operator from identical states:
    rho, phi, gradients, particles and tallies agree with the oracle."""
    cfg = workload(n1=64, n2=32, alpha=0.15, B=0.5, n_init=20000, precision="fp64", no_inject=True,
                   poisson_tol=1e-13, poisson_max_iter=60, fe_operator=True)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp, seed, vs in ((0, 11, 1.0), (1, 12, 0.03)):
        st = random_states(20000, cfg["x1_out"], seed=seed, vscale=vs)
        s.add_particles(sp, st)
        o.add_particles(sp, st)
    s.step(1)
    o.step(1)
    assert rel(s.field("rho"), o.grid("rho")) < 1e-11
    assert rel(s.field("phi"), o.grid("phi")) < 1e-11
    assert rel(s.field("G1"), o.grid("G1")) < 1e-9
    for sp in (0, 1):
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape
        assert np.abs(g - r).max() < 1e-9
        assert s.tallies()["counts"][sp]["absorbed"] == o.counts()[sp]["absorbed"]
    assert rel(s.tallies()["bins"], o.bins()) < 1e-9


def test_fe_with_isolated_grain_matches_oracle(apic):
    """The conservative operator under the isolated grain's correction: four
    FP64 steps agree with the oracle (grain potential, charge, phi, particles)."""
    cfg = workload(n1=48, n2=24, alpha=-0.2, B=0.5, n_init=10000, precision="fp64", no_inject=True,
                   phi_g=-0.5, poisson_tol=1e-13, poisson_max_iter=60, floating=True, fe_operator=True)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp, seed, vs in ((0, 41, 1.0), (1, 42, 0.03)):
        st = random_states(10000, cfg["x1_out"], seed=seed, vscale=vs)
        s.add_particles(sp, st)
        o.add_particles(sp, st)
    s.step(4)
    o.step(4)
    hg, ho = s.tallies(history=True)["history"], o.history()
    assert np.abs(hg[:, 10] - ho[:, 10]).max() < 1e-9
    assert abs(ho[-1, 10] - ho[0, 10]) > 1e-3
    assert rel(s.field("phi"), o.grid("phi")) < 1e-10
    for sp in (0, 1):
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape and np.abs(g - r).max() < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fe_with_boltzmann_electrons_matches_oracle(apic, precision):
    """The Newton solve of Boltzmann electrons on the conservative operator."""
    from tests.inputs import ION
    cfg = dict(alpha=0.15, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, B=0.0, dt=0.5, n1=64, n2=32,
               species=[dict(ION, n_init=20000)], no_inject=True, boltzmann=True, fe_operator=True,
               precision=precision, poisson_tol=1e-12, poisson_max_iter=80, newton_iters=12, seed=3)
    rho = 1.0 + 0.3 * random_rho(64, 32, seed=17)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    assert rel(s.solve_poisson(rho), o.solve(rho)) < 1e-9
