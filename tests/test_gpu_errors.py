"""Error paths of the C ABI (include/apic.h).  Each error is produced by the
inputs or by a bounded device wait running out, never by a GPU fault: a
particle capacity too small for the load or for the injected particles, a
Poisson iteration limit too small for the tolerance, a NaN in a given charge
density, and a grid-barrier wait that nothing completes.  Errors are sticky
on their object; other objects and the CUDA context stay usable."""
import time

import numpy as np
import pytest

from tests.inputs import random_rho, workload

pytestmark = pytest.mark.gpu

CAPACITY, NOT_CONVERGED, NONFINITE, TIMEOUT = -3, -4, -5, -6


@pytest.fixture(scope="module")
def apic():
    import torch

    import paper_2307_11107_gb300 as apic
    apic.build()
    torch.cuda.set_device(0)
    return apic


def _code(fn):
    from paper_2307_11107_gb300.sim import ApicError
    try:
        fn()
    except ApicError as e:
        return e.code
    return 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_capacity_on_load(apic, prec):
    cfg = workload(n1=32, n2=16, n_init=4000, precision=prec)
    cfg["species"] = [dict(sp, capacity=2048) for sp in cfg["species"]]
    s = apic.Sim(cfg)
    assert _code(lambda: s.load_volume(0, 4000)) == CAPACITY
    s.load_volume(0, 2000)  # a load that fits still works (the host check rejects before any work)
    s.step(1)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_capacity_during_injection(apic, prec):
    """An empty domain whose per-step surface injection (about 1200 electrons
    at this macro-weight) exceeds the 1024 slots: the injection kernel sets
    the capacity bit, apic_step returns CAPACITY and keeps returning it."""
    cfg = workload(n1=32, n2=16, n_init=100000, precision=prec)
    cfg["species"] = [dict(sp, capacity=1024) for sp in cfg["species"]]
    s = apic.Sim(cfg)
    assert _code(lambda: s.step(1)) == CAPACITY
    assert _code(lambda: s.step(1)) == CAPACITY  # sticky
    assert _code(lambda: s.tallies()) == CAPACITY
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_not_converged(apic, prec):
    """One iteration (one refinement pass of the FP32 direct solve, or one
    BiCGSTAB iteration with a multigrid cycle) cannot reach a relative
    residual of 1e-15.  (128 x 64 cells: on smaller grids the multigrid's
    coarsest level, a dense inverse, is the whole grid and one iteration is
    exact.)"""
    cfg = workload(n1=128, n2=64, alpha=0.15, precision=prec, poisson_tol=1e-15, poisson_max_iter=1)
    s = apic.Sim(cfg)
    rho = random_rho(128, 64, seed=3)
    assert _code(lambda: s.solve_poisson(rho)) == NOT_CONVERGED
    s.close()
    ok = apic.Sim(dict(cfg, poisson_tol=1e-10, poisson_max_iter=20))
    phi = ok.solve_poisson(rho)
    assert np.isfinite(phi).all()
    ok.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonfinite_density(apic, prec):
    cfg = workload(n1=64, n2=32, alpha=0.15, precision=prec)
    s = apic.Sim(cfg)
    rho = random_rho(64, 32, seed=4)
    rho[20, 7] = np.nan
    assert _code(lambda: s.solve_poisson(rho)) == NONFINITE
    s.close()


def test_grid_barrier_wait_runs_out(apic):
    """The grid barrier of the cooperative solvers gives up after its time
    limit: four CTAs wait at a barrier that expects a fifth arrival, each
    stops after 50 ms, and the object reports TIMEOUT.  A new object then
    steps normally on the same context."""
    cfg = workload(n1=32, n2=16, n_init=2000, precision="fp64")
    s = apic.Sim(cfg)
    t0 = time.perf_counter()
    assert s.check_wait_limit(50_000_000) == TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    assert _code(lambda: s.step(1)) == TIMEOUT  # sticky
    s.close()
    s2 = apic.Sim(cfg)
    for sp in (0, 1):
        s2.load_volume(sp, 2000)
    s2.step(2)
    assert s2.tallies()["step"] == 2
    s2.close()
