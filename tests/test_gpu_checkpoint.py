"""Checkpoint and resume: a run continued from a checkpoint (in the same object
or in a new one created with the same configurations) gives the tallies,
fields and particle set of the uninterrupted run bit for bit, because every
random draw is a counter-based Philox draw of the saved draw count."""
import numpy as np
import pytest

from tests.inputs import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import torch
    import paper_2307_11107_gb300 as apic
    assert torch.cuda.is_available()
    apic.build()
    return apic


def _cfgs(prec):
    base = dict(precision=prec, sort_interval=3, x1_out=-0.1, history_cap=64)
    return [
        workload(n1=64, n2=32, alpha=0.1, phi_g=-2.0, B=1.0, n_init=20000, seed=3, instance=0, **base),
        workload(n1=96, n2=48, alpha=-0.2, phi_g=-3.0, B=0.0, n_init=12000, seed=3, instance=1, **base),
    ]


def _state(s, cfgs):
    out = []
    for k in range(len(cfgs)):
        t = s.tallies(k)
        parts = [s.particles(sp, instance=k) for sp in (0, 1)]
        parts = [p[np.lexsort(p.T[::-1])] for p in parts]
        out.append((t, s.field("phi", instance=k), s.field("rho", instance=k), parts))
    return out


def _same(a, b):
    for (ta, pa, ra, qa), (tb, pb, rb, qb) in zip(a, b):
        assert ta["step"] == tb["step"]
        assert ta["counts"] == tb["counts"]
        assert np.array_equal(ta["bins"], tb["bins"])
        assert np.array_equal(ta["history"], tb["history"])
        assert np.array_equal(pa, pb) and np.array_equal(ra, rb)
        for x, y in zip(qa, qb):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_resume_from_checkpoint_is_exact(apic, prec):
    cfgs = _cfgs(prec)
    s = apic.Sim(cfgs)
    for k, c in enumerate(cfgs):
        for sp in range(len(c["species"])):
            s.load_volume(sp, c["species"][sp]["n_init"], instance=k)
    s.step(7)
    ck = s.checkpoint()
    s.step(5)
    ref = _state(s, cfgs)
    # the same object, rewound
    s.restore(ck)
    assert s.tallies(0)["step"] == 7
    s.step(5)
    _same(_state(s, cfgs), ref)
    # a new object with the same configurations
    t = apic.Sim(cfgs)
    t.restore(ck)
    t.step(5)
    _same(_state(t, cfgs), ref)
    # refused: another layout, a truncated or altered buffer; the object stays usable
    u = apic.Sim([cfgs[0]])
    with pytest.raises(RuntimeError):
        u.restore(ck)
    with pytest.raises(RuntimeError):
        t.restore(ck[: len(ck) // 2])
    bad = ck.copy()
    bad[:8] = 0
    with pytest.raises(RuntimeError):
        t.restore(bad)
    t.step(1)
    assert t.tallies(0)["step"] == 13
    for x in (s, t, u):
        x.close()
