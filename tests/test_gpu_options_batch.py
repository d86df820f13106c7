"""The options side by side: one batch whose instances use different ones
(isolated grain with the conservative operator, Boltzmann electrons, chord
absorption, none) computes what each instance computes alone on the same
kernels (per-phase multigrid, which the Boltzmann instance requires)."""
import os

import numpy as np
import pytest

from tests.inputs import ELECTRON, ION

pytestmark = pytest.mark.gpu


def _cfgs():
    base = dict(alpha=0.12, x1_out=-0.1, phi_g=-1.5, phi_out=0.0, B=0.5, dt=0.2, n1=32, n2=16, seed=6,
                precision="fp64", poisson_tol=1e-12, poisson_max_iter=80)
    two = [dict(ELECTRON, n_init=8000), dict(ION, n_init=8000)]
    return [dict(base, species=two, floating=True, fe_operator=True, instance=0),
            dict(base, species=[dict(ION, n_init=8000)], boltzmann=True, newton_iters=10, instance=1),
            dict(base, species=two, chord_absorb=True, dt=0.5, instance=2),
            dict(base, species=two, instance=3, alpha=-0.2, n1=48, n2=24)]


def _run(apic, cfgs, steps):
    s = apic.Sim(cfgs)
    for k, c in enumerate(cfgs):
        for sp in range(len(c["species"])):
            s.load_volume(sp, c["species"][sp]["n_init"], instance=k)
    s.step(steps)
    out = []
    for k, c in enumerate(cfgs):
        parts = [s.particles(sp, instance=k) for sp in range(len(c["species"]))]
        out.append((s.field("phi", k), parts, s.tallies(k, history=True)))
    s.close()
    return out


def test_mixed_options_batch_equals_solo(monkeypatch):
    import paper_2307_11107_gb300 as apic
    apic.build()
    monkeypatch.setenv("APIC_PRECOND", "mg")
    monkeypatch.setenv("APIC_SOLVER", "kernels")
    cfgs = _cfgs()
    batched = _run(apic, cfgs, 5)
    for k, c in enumerate(cfgs):
        (pb, qb, tb), = [batched[k]]
        (ps, qs, ts), = _run(apic, [c], 5)
        assert np.array_equal(pb, ps), k
        for a, b in zip(qb, qs):
            assert a.shape == b.shape
            assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
        assert tb["counts"] == ts["counts"]
        assert np.allclose(tb["history"], ts["history"], rtol=1e-12, atol=1e-12)
    # the options did something: the isolated grain's potential moved
    h0 = batched[0][2]["history"]
    assert h0[-1, 10] != h0[0, 10]
