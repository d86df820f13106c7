"""GPU path (libapic.so on sm_103a) against the FP64 CPU oracle, element by
element on identical seeded inputs."""
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
@pytest.mark.parametrize("grid", [(64, 32), (96, 48)])
def test_node_volumes(apic, alpha, grid):
    cfg = workload(n1=grid[0], n2=grid[1], alpha=alpha, n_init=1000, precision="fp64")
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    assert rel(s.field("V"), o.grid("V")) < 1e-12


@pytest.mark.parametrize("alpha", [0.0, 0.15, 0.225, -0.24])
@pytest.mark.parametrize("grid", [(64, 32), (128, 64), (256, 128)])
def test_poisson_fp64_matches_banded_lu(apic, alpha, grid):
    """GPU BiCGSTAB + multigrid (FP64) reproduces the oracle's LU solution of Eqs. 6-7."""
    n1, n2 = grid
    cfg = workload(n1=n1, n2=n2, alpha=alpha, x1_out=-0.05, n_init=1000, precision="fp64",
                   poisson_tol=1e-13, poisson_max_iter=60)
    rho = random_rho(n1, n2, seed=n1 + 7, scale=0.3)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    assert rel(s.solve_poisson(rho), o.solve(rho)) < 1e-10


@pytest.mark.parametrize("direct", ["bcr", "nd"])
@pytest.mark.parametrize("alpha,grid", [(0.15, (256, 128)), (0.225, (256, 128)), (0.15, (96, 48)),
                                        (0.225, (288, 144)), (-0.24, (160, 80)), (0.15, (64, 300)),
                                        (0.225, (32, 512))])
def test_poisson_fp32_refined_matches_banded_lu(apic, alpha, grid, direct, monkeypatch):
    """The FP32 direct solve inside the FP64 residual loop reaches the FP64
    solution: the block cyclic reduction (n1 a power of two and not, rows
    beyond n1 - 1 padded with a zero correction; blocks wider than 256
    unknowns in the wide kernel) and the nested-dissection factorisation."""
    monkeypatch.setenv("APIC_DIRECT", direct)
    n1, n2 = grid
    cfg = workload(n1=n1, n2=n2, alpha=alpha, x1_out=-0.05, n_init=1000, precision="fp32",
                   poisson_tol=1e-12, poisson_max_iter=60)
    rho = random_rho(n1, n2, seed=n1 + 3, scale=0.3)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    assert s.stats()["solver"].startswith("FP32 block cyclic reduction" if direct == "bcr" else "FP32 nested dissection")
    assert rel(s.solve_poisson(rho), o.solve(rho)) < 1e-9


@pytest.mark.parametrize("alpha,grid", [(0.225, (16, 1024)), (-0.24, (24, 640))])
def test_poisson_nested_dissection_beyond_reduction_width(apic, alpha, grid):
    """Grids wider than the block cyclic reduction takes (543 cells in x2)
    are solved by the nested dissection to the same accuracy."""
    n1, n2 = grid
    cfg = workload(n1=n1, n2=n2, alpha=alpha, x1_out=-0.05, n_init=1000, precision="fp32",
                   poisson_tol=1e-12, poisson_max_iter=60)
    rho = random_rho(n1, n2, seed=n1 + 5, scale=0.3)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    assert s.stats()["solver"].startswith("FP32 nested dissection")
    assert rel(s.solve_poisson(rho), o.solve(rho)) < 1e-9


@pytest.mark.parametrize("alpha,B", [(0.0, 0.0), (0.15, 1.0), (-0.24, 0.5)])
def test_single_step_fp64(apic, alpha, B):
    """One full step from identical explicit states (no injection): rho, phi,
    node gradients, every surviving particle and the tallies (with a binding
    energy for absorbed ions) agree with the oracle."""
    cfg = workload(n1=64, n2=32, alpha=alpha, B=B, n_init=20000, precision="fp64", no_inject=True,
                   poisson_tol=1e-13, poisson_max_iter=60, e_bind_ion=2.0)
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
    t = s.tallies()
    for sp in (0, 1):
        assert t["counts"][sp]["absorbed"] == o.counts()[sp]["absorbed"]
        assert t["counts"][sp]["escaped"] == o.counts()[sp]["escaped"]
    assert rel(t["bins"], o.bins()) < 1e-9


@pytest.mark.parametrize("alpha", [0.0, 0.15])
def test_volume_load_matches_oracle(apic, alpha):
    cfg = workload(n1=32, n2=16, alpha=alpha, n_init=30000, precision="fp64", seed=5)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, 30000)
        o.load_volume(sp, 30000)
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape
        assert np.abs(g - r).max() < 1e-12


def test_surface_injection_matches_oracle(apic):
    """Per-step injection (Eq. 4 sampling, half-Maxwellian, free flight): the
    set of injected particles equals the oracle's (the GPU stores them in
    scheduling order, so rows are compared after sorting)."""
    cfg = workload(n1=32, n2=16, alpha=0.15, n_init=4000, precision="fp64", seed=9, no_field=True)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    s.step(3)
    o.step(3)
    for sp in (0, 1):
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape
        gi, ri = np.lexsort(g.T[::-1]), np.lexsort(r.T[::-1])
        assert np.abs(g[gi] - r[ri]).max() < 1e-12
        c = s.tallies()["counts"][sp]
        assert c["injected"] == o.counts()[sp]["injected"]


@pytest.mark.slow
def test_spherical_200_steps_fp64(apic):
    """Spherical grain, 64 x 32 cells, 1e5 per species, 200 steps, FP64 on both
    sides: fields within 1e-5 and cumulative tallies within 1e-4."""
    from paper_2307_11107_gb300.workloads import spherical_small
    cfg = spherical_small("fp64")
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, 100000)
        o.load_volume(sp, 100000)
    s.step(200)
    o.step(200)
    assert rel(s.field("rho"), o.grid("rho")) < 1e-5
    assert rel(s.field("phi"), o.grid("phi")) < 1e-5
    t = s.tallies()
    ob = o.bins()
    for sp in (0, 1):
        tot_g, tot_o = t["bins"][sp].sum(axis=0), ob[sp].sum(axis=0)
        assert np.all(np.abs(tot_g - tot_o) <= 1e-4 * np.abs(tot_o) + 1e-12), (sp, tot_g, tot_o)
    h, ho = t["history"], o.history()
    assert h.shape == ho.shape
    assert np.allclose(h[:, 3], ho[:, 3], rtol=1e-5, atol=1e-8)
    assert np.allclose(h[:, 6], ho[:, 6], rtol=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sorting_does_not_change_results(apic, prec):
    """Sorting by cell (and compaction of freed slots) only reorders
    particles: integer deposit sums, fixed-order reductions and per-particle
    pushes make rho and phi bit-identical and the particle sets equal, and the
    fixed-point tallies make the bins and the history's tallies bit-identical."""
    cfg = workload(n1=64, n2=32, alpha=0.15, B=1.0, n_init=40000, precision=prec, seed=4)
    runs = []
    for si in (0, 3):
        s = apic.Sim(dict(cfg, sort_interval=si))
        for sp in (0, 1):
            s.load_volume(sp, 40000)
        s.step(10)
        runs.append((s.field("rho"), s.field("phi"), [s.particles(sp) for sp in (0, 1)], s.tallies()))
    (r0, p0, q0, t0), (r1, p1, q1, t1) = runs
    assert np.array_equal(r0, r1) and np.array_equal(p0, p1)
    for a, b in zip(q0, q1):
        assert a.shape == b.shape
        assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
    for sp in (0, 1):
        assert t0["counts"][sp] == t1["counts"][sp]
    # fixed-point tallies: the bins and the step history do not depend on the
    # order in which the absorption events arrive
    assert np.array_equal(t0["bins"], t1["bins"])
    assert np.array_equal(t0["history"][:, [1, 2, 4, 5, 9]], t1["history"][:, [1, 2, 4, 5, 9]])


def test_fp32_fma_probe(apic):
    """The FP32 CUDA-core ceiling the push's arithmetic is compared with: the
    probe runs and reports a plausible GB300 figure (152 SMs x 128 lanes x 2
    FLOPs at up to 2.07 GHz is about 80 TFLOP/s)."""
    t = apic.probe_fp32_fma()
    assert 20.0 < t < 100.0, t
