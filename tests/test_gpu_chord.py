"""Chord-intersection absorption (an option beside the paper's end-point test
of Sec. 2): the GPU path against the FP64 oracle with the option on, on steps
long enough that many straight chords cross the grain between end points."""
import numpy as np
import pytest

import oracle
from tests.inputs import random_states, workload

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


def _cfg(alpha, B, precision, chord=True, **kw):
    return workload(n1=64, n2=32, alpha=alpha, B=B, dt=0.5, n_init=20000, precision=precision,
                    no_inject=True, poisson_tol=1e-13, poisson_max_iter=60,
                    chord_absorb=chord, **kw)


def _load(sims, cfg, vs=3.0):
    for sp, seed, v in ((0, 11, vs), (1, 12, 0.03 * vs)):
        st = random_states(20000, cfg["x1_out"], seed=seed, vscale=v)
        for s in sims:
            s.add_particles(sp, st)


@pytest.mark.parametrize("alpha,B", [(0.0, 0.0), (0.15, 0.5), (-0.24, 1.0)])
def test_chord_single_step_fp64(apic, alpha, B):
    """One FP64 step with the option: absorbed and escaped counts equal the
    oracle's, the surviving particles and the polar-angle bins agree, and the
    option really changes the outcome (the oracle without it absorbs fewer)."""
    cfg = _cfg(alpha, B, "fp64", e_bind_ion=2.0)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    plain = oracle.Sim(_cfg(alpha, B, "fp64", chord=False, e_bind_ion=2.0))
    _load((s, o, plain), cfg)
    s.step(1)
    o.step(1)
    plain.step(1)
    t = s.tallies()
    for sp in (0, 1):
        assert t["counts"][sp]["absorbed"] == o.counts()[sp]["absorbed"]
        assert t["counts"][sp]["escaped"] == o.counts()[sp]["escaped"]
        g, r = s.particles(sp), o.particles(sp)[0]
        assert g.shape == r.shape
        assert np.abs(g - r).max() < 1e-9
    assert rel(t["bins"], o.bins()) < 1e-9
    assert o.counts()[0]["absorbed"] > plain.counts()[0]["absorbed"] + 100


def test_chord_single_step_fp32_counts(apic):
    """FP32 push with the option: the absorbed count is within a few parts in
    a thousand of the FP64 oracle's (orbits that graze the grain can go either
    way in single precision)."""
    cfg = _cfg(0.15, 0.5, "fp32")
    s, o = apic.Sim(cfg), oracle.Sim(dict(cfg, precision="fp64"))
    _load((s, o), cfg)
    s.step(1)
    o.step(1)
    t = s.tallies()
    for sp in (0, 1):
        a, b = t["counts"][sp]["absorbed"], o.counts()[sp]["absorbed"]
        assert abs(a - b) <= max(3, 3e-3 * b), (sp, a, b)


def test_chord_injection_fp64(apic):
    """Injection with the option (the partial first step of an injected
    particle takes the same chord test): the set of particles after three
    field-free steps equals the oracle's."""
    cfg = workload(n1=32, n2=16, alpha=0.15, dt=0.5, n_init=4000, precision="fp64", seed=9,
                   no_field=True, chord_absorb=True)
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
        assert c["absorbed"] == o.counts()[sp]["absorbed"]


def test_chord_rejected_by_sensitivity(apic):
    """The tangent (adjoint) step has no derivative of the chord test, so the
    sensitivity entry point refuses a configuration that enables it."""
    cfg = _cfg(0.15, 0.0, "fp64")
    s = apic.Sim(cfg)
    _load((s,), cfg)
    with pytest.raises(apic.ApicError, match="CHORD"):
        s.sensitivity(2)
