"""Batched form: several uneven instances (different alpha, grain potential,
B, grid and particle counts) advance together in every launch.  Each instance
of the batch must compute exactly what it computes alone."""
import numpy as np
import pytest

from tests.inputs import workload

pytestmark = pytest.mark.gpu


def _instances(prec):
    base = dict(precision=prec, sort_interval=3, x1_out=-0.1)
    return [
        workload(n1=64, n2=32, alpha=0.1, phi_g=-2.0, B=0.0, n_init=20000, seed=2, instance=0, **base),
        workload(n1=96, n2=48, alpha=0.2, phi_g=-3.5, B=1.0, n_init=8000, seed=2, instance=1, **base),
        workload(n1=128, n2=64, alpha=-0.24, phi_g=-1.0, B=1.0, n_init=30000, seed=2, instance=2, **base),
    ]


_SOLVER = {"bcr": "FP32 block cyclic reduction", "nd": "FP32 nested dissection",
           "mg": "multigrid BiCGSTAB, per-phase kernels"}


def _run(apic, cfgs, steps, solver=None):
    s = apic.Sim(cfgs)
    if solver is not None:
        assert s.stats()["solver"].startswith(_SOLVER[solver])
    for k, c in enumerate(cfgs):
        for sp in range(len(c["species"])):
            s.load_volume(sp, c["species"][sp]["n_init"], instance=k)
    s.step(steps)
    out = []
    for k in range(len(cfgs)):
        parts = [s.particles(sp, instance=k) for sp in (0, 1)]
        out.append((s.field("rho", k), s.field("phi", k), parts, s.tallies(k)))
    s.close()
    return out


@pytest.mark.parametrize("prec,solver", [("fp64", "mg"), ("fp32", "bcr"), ("fp32", "nd"), ("fp32", "mg")])
def test_batch_equals_solo(prec, solver, monkeypatch):
    """Same solver path for the batch and each instance alone (the block
    cyclic reduction or the nested dissection of every instance in one
    launch, or the per-phase multigrid kernels): the results agree bit for
    bit."""
    import paper_2307_11107_gb300 as apic
    apic.build()
    cfgs = _instances(prec)
    if solver == "mg":
        monkeypatch.setenv("APIC_PRECOND", "mg")
    if solver in ("bcr", "nd"):
        monkeypatch.setenv("APIC_DIRECT", solver)
    batched = _run(apic, cfgs, 6, solver)
    if solver == "mg":
        monkeypatch.setenv("APIC_SOLVER", "kernels")
    for k, c in enumerate(cfgs):
        (rb, pb, qb, tb), = [batched[k]]
        (rs, ps, qs, ts), = _run(apic, [c], 6, solver)
        assert np.array_equal(rb, rs)
        assert np.array_equal(pb, ps)
        for a, b in zip(qb, qs):
            assert a.shape == b.shape
            assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
        for sp in (0, 1):
            assert tb["counts"][sp] == ts["counts"][sp]
        assert np.array_equal(tb["bins"], ts["bins"])
        assert np.allclose(tb["history"], ts["history"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("direct", ["bcr", "auto", "wide"])
def test_batched_reduction_poisson_matches_banded_lu(direct, monkeypatch):
    """Every instance of an uneven FP32 batch (different alpha and grid, n1
    a power of two or not, one instance wider than 256 unknowns per row, so
    the wide kernel runs the narrow ones too) solved by the batched block
    cyclic reduction against the oracle's banded LU; by default (the
    reduction would not fit in L2) every instance takes the nested
    dissection; with APIC_DIRECT=wide the wide instance takes it in the same
    launch as the others' reduction.  Solving one instance leaves the
    others' potential alone."""
    import oracle
    import paper_2307_11107_gb300 as apic
    from tests.inputs import random_rho
    apic.build()
    monkeypatch.setenv("APIC_DIRECT", direct)
    grids = [(64, 32, 0.1), (96, 48, 0.2), (160, 80, -0.24), (256, 128, 0.15), (32, 300, 0.05)]
    cfgs = [workload(n1=a, n2=b, alpha=al, x1_out=-0.05, n_init=1000, precision="fp32", poisson_tol=1e-12,
                     poisson_max_iter=60, instance=k) for k, (a, b, al) in enumerate(grids)]
    s = apic.Sim(cfgs)
    assert s.stats()["solver"].startswith(_SOLVER["bcr" if direct == "bcr" else "nd"])
    before = [s.field("phi", k) for k in range(len(cfgs))]
    for k, c in enumerate(cfgs):
        rho = random_rho(c["n1"], c["n2"], seed=40 + k, scale=0.3)
        ref = oracle.Sim(c).solve(rho)
        got = s.solve_poisson(rho, instance=k)
        assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-9
    for k in range(len(cfgs)):
        assert np.array_equal(s.field("phi", k), before[k])
    s.close()


def test_set_schedule_applies_and_leaves_results_unchanged():
    """A schedule applied by apic_set_schedule is the one in use (the stats
    report it, and timed steps time their sorts), out-of-range values are
    refused, and the fixed-point deposits and tallies make the results
    bit-identical to those of the default schedule."""
    import paper_2307_11107_gb300 as apic
    apic.build()
    cfgs = _instances("fp32")
    runs = []
    for sched in (None, (2, 4, 2, 32)):
        s = apic.Sim(cfgs)
        for k, c in enumerate(cfgs):
            for sp in range(len(c["species"])):
                s.load_volume(sp, c["species"][sp]["n_init"], instance=k)
        s.step(3)
        if sched is not None:
            for bad in ((-1, 0, 0, 0), (0, 1, 0, 0), (0, 17, 0, 0), (0, 0, 65, 0), (0, 0, 0, 24)):
                with pytest.raises(RuntimeError):
                    s.set_schedule(*bad)
            s.set_schedule(*sched)
            st = s.stats()
            assert (st["sort_interval"], st["win_rows"], st["chunk_group"], st["chunk_items"]) == sched
        s.step(4)
        s.step_timed(4)
        st = s.stats()
        si = st["sort_interval"]
        assert st["timed_sorts"] == sum(1 for k in range(7, 11) if k % si == 0)
        assert (st["sort_ms"] > 0.0) == (st["timed_sorts"] > 0)
        runs.append([s.tallies(k) for k in range(len(cfgs))] + [s.field("phi", instance=k) for k in range(len(cfgs))])
        s.close()
    a, b = runs
    for k in range(len(cfgs)):
        assert np.array_equal(a[k]["bins"], b[k]["bins"])
        assert a[k]["counts"] == b[k]["counts"]
        assert np.array_equal(a[k]["history"][:, [1, 2, 4, 5, 9]], b[k]["history"][:, [1, 2, 4, 5, 9]])
        assert np.array_equal(a[len(cfgs) + k], b[len(cfgs) + k])


def test_autotune_keeps_a_candidate_and_stepping_stays_valid():
    """The autotuner times every sort interval, keeps the fastest, tunes the
    push's tiles at it and leaves a simulation that steps on with consistent
    counts."""
    import paper_2307_11107_gb300 as apic
    apic.build()
    cfgs = _instances("fp32")
    s = apic.Sim(cfgs)
    for k, c in enumerate(cfgs):
        for sp in range(len(c["species"])):
            s.load_volume(sp, c["species"][sp]["n_init"], instance=k)
    s.step(4)
    chosen, ms = s.autotune(4)
    assert chosen in ms and all(v > 0.0 for v in ms.values())
    assert ms[chosen] == min(ms.values())
    st = s.stats()
    assert st["sort_interval"] == chosen
    assert st["chunk_group"] in (2, 4, 8) and st["win_rows"] in (2, 4, 6, 8, 12, 16) and st["chunk_items"] in (16, 32)
    s.step(5)
    for k in range(len(cfgs)):
        t = s.tallies(k)
        # each interval candidate runs whole intervals, c * ceil(4 / c) steps;
        # each of the 3 + 6 + 2 tile candidates one warm-up interval and as many
        tiles = 11 * (chosen + chosen * -(-4 // chosen))
        assert t["step"] == 4 + sum(c * -(-4 // c) for c in ms) + tiles + 5
        for sp in (0, 1):
            cnt = t["counts"][sp]
            assert cnt["resident"] == s.particles(sp, instance=k).shape[0]
    s.close()
