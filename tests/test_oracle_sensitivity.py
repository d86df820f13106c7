"""Pins of the oracle's frozen-decision finite differences (the reference for
the sensitivity window): replay fidelity, the structure the frozen decisions
impose, and closed forms of the vacuum sphere (Gauss's law, mirror symmetry
of the shape family of Eq. 2)."""
import numpy as np
import pytest

import oracle
from oracle.sensitivity import PARAMS, window_outputs, window_sensitivity
from tests.inputs import random_states, workload


def _states(n, x1_out, seed):
    return [random_states(n, x1_out, seed=seed), random_states(n, x1_out, seed=seed + 1, vscale=0.03)]


def _cfg(**kw):
    d = dict(n1=32, n2=16, alpha=0.15, B=0.5, n_init=4000, x1_out=-0.1, seed=3)
    d.update(kw)
    return workload(**d)


def test_replay_reproduces_the_recorded_run():
    cfg = _cfg()
    st = _states(4000, cfg["x1_out"], 11)
    runs = []
    for mode in ("record", "replay"):
        s = oracle.Sim(cfg)
        for sp in (0, 1):
            s.add_particles(sp, st[sp])
        if mode == "replay":
            s.set_tape(tape)
            s.tape_mode(s.TAPE_REPLAY)
        else:
            s.tape_mode(s.TAPE_RECORD)
        s.step(6)
        if mode == "record":
            tape = s.tape()
        runs.append(s)
    a, b = runs
    assert b.tape_ok()
    assert np.array_equal(a.history(), b.history())
    for sp in (0, 1):
        assert np.array_equal(a.particles(sp)[0], b.particles(sp)[0])
    # one status per particle update and injection draw, one count per step and species
    c = a.counts()
    assert tape[1].size == 6 * 2
    assert tape[0].size >= 6 * 2 * 4000 - sum(x["absorbed"] + x["escaped"] for x in c)


def test_frozen_decisions_fix_the_current():
    """With every absorption held, the current is q w (events) / dt: it cannot
    move with phi_g or B, and moves with alpha only through w = V_dom / N."""
    cfg = _cfg()
    st = _states(4000, cfg["x1_out"], 21)
    K = 5
    vals, jac, _ = window_sensitivity(cfg, st, K)
    assert vals[2] != 0.0
    assert jac[2, 1] == 0.0 and jac[2, 2] == 0.0
    h = 1e-6
    vp = oracle.Sim(dict(cfg, alpha=cfg["alpha"] + h)).scalars()["V_dom"]
    vm = oracle.Sim(dict(cfg, alpha=cfg["alpha"] - h)).scalars()["V_dom"]
    dlnw = (np.log(vp) - np.log(vm)) / (2 * h)
    # d ln w / d alpha is ~1e-5 here: both sides carry the rounding of a
    # difference of nearly equal sums over h (about 1e-4 relative)
    assert jac[2, 0] == pytest.approx(vals[2] * dlnw, rel=1e-4)


def test_central_differences_converge():
    """Frozen decisions make the window a smooth function of the parameters:
    the central differences at h and 2h agree to second order."""
    cfg = _cfg()
    st = _states(4000, cfg["x1_out"], 31)
    K = 5
    _, j1, _ = window_sensitivity(cfg, st, K, h=dict(alpha=2e-6, phi_g=2e-6, B=2e-6))
    _, j2, _ = window_sensitivity(cfg, st, K, h=dict(alpha=4e-6, phi_g=4e-6, B=4e-6))
    scale = np.abs(j1).max(axis=1, keepdims=True) + 1e-30
    assert (np.abs(j1 - j2) / scale).max() < 1e-4


def test_vacuum_sphere_gauss_law_and_symmetry():
    """No particles, alpha = 0: phi is linear in x1 (1/r is harmonic), so the
    discrete solution is exact and Q = 4 pi (phi_g - phi_out) / (1 + x1_out):
    dQ/dphi_g = 4 pi / (1 + x1_out).  The shape family is mirror-symmetric
    (alpha -> -alpha with x2 -> -x2): dQ/dalpha = 0, and F_Z = 0 for every
    phi_g, so dF_Z/dphi_g = 0."""
    cfg = _cfg(alpha=0.0, no_inject=True)
    vals, jac, _ = window_sensitivity(cfg, [None, None], 3)
    x1o = cfg["x1_out"]
    assert vals[4] == pytest.approx(4 * np.pi * (cfg["phi_g"] - cfg["phi_out"]) / (1 + x1o), rel=1e-12)
    assert jac[4, 1] == pytest.approx(4 * np.pi / (1 + x1o), rel=1e-7)
    assert abs(jac[4, 0]) < 1e-6 * abs(vals[4])
    assert vals[1] == pytest.approx(0.0, abs=1e-12) and abs(jac[1, 1]) < 1e-8
    assert np.all(jac[[0, 2, 3]] == 0.0)  # no particles, nothing absorbed
    assert np.all(jac[:, 2] == 0.0)       # B acts on particles only


def test_outputs_are_the_history_columns():
    cfg = _cfg()
    s = oracle.Sim(cfg)
    st = _states(2000, cfg["x1_out"], 41)
    for sp in (0, 1):
        s.add_particles(sp, st[sp])
    s.step(4)
    h = s.history()
    v = window_outputs(s, 4)
    assert v[0] == pytest.approx(h[:, 2].mean()) and v[2] == pytest.approx(h[:, 1].mean())
    assert PARAMS == ("alpha", "phi_g", "B")


def test_frozen_cells_make_the_differences_converge():
    """Enough particles that many cross a cell boundary within +-h: with each
    particle's cell and each injection's table interval replayed (bilinear
    weights continued, not switched), the replayed map is smooth and the
    central differences converge at O(h^2): the change from h = 1e-4 to 1e-5
    is about 100 times the change from 1e-5 to 1e-6, on every output row
    (the current's row, rounding-limited, excepted)."""
    n, K = 40000, 4
    cfg = workload(n1=64, n2=32, alpha=0.15, B=1.0, x1_out=-0.05, n_init=n, Ti=0.5, seed=5)
    st = [random_states(n, cfg["x1_out"], seed=81), random_states(n, cfg["x1_out"], seed=82, vscale=0.0165)]
    J = [window_sensitivity(cfg, st, K, h=dict(alpha=h, phi_g=h, B=h))[1] for h in (1e-4, 1e-5, 1e-6)]
    rows = [0, 1, 3, 4]
    scale = np.abs(J[2][rows]).max(axis=1, keepdims=True)
    d1 = np.abs(J[0][rows] - J[1][rows]) / scale
    d2 = np.abs(J[1][rows] - J[2][rows]) / scale
    assert d2.max() < 1e-5, d2
    assert d1.max() < 1e-2, d1
    # replaying the recorded cells leaves the unperturbed run unchanged
    base = oracle.Sim(cfg)
    for sp in (0, 1):
        base.add_particles(sp, st[sp])
    base.tape_mode(base.TAPE_RECORD)
    base.step(K)
    tape = base.tape()
    again = oracle.Sim(cfg)
    for sp in (0, 1):
        again.add_particles(sp, st[sp])
    again.set_tape(tape)
    again.tape_mode(again.TAPE_REPLAY)
    again.step(K)
    assert again.tape_ok()
    assert np.array_equal(base.history(), again.history())
