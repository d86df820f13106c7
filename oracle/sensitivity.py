"""Frozen-decision finite differences of the oracle (test infrastructure only).

The window outputs of the step (drag F_Z = absorbed Z momentum per time,
electric F_Z on the grain, current = absorbed charge per time, torque T_z =
absorbed L_z per time, grain charge Q; history columns 2, 3, 1, 4, 6 of the
oracle) are averaged over a window of K steps that starts from a given
particle state.  Their derivatives with respect to alpha, phi_g and B are
central differences of runs at p +- h that replay the decisions of the run at
p (absorbed, escaped or kept, per update and per injection draw; injection
counts; every particle's cell at every weighing and gather, whose bilinear
weights are then taken unclamped; every injection's sampling-table
interval), so that no particle changes fate or piece of the piecewise
bilinear weights between the runs: the replayed map is smooth in the
parameters and its central differences converge at O(h^2) to the
frozen-decision derivative.  Random numbers are the same in every run (same
seed and draw counters).
"""
import numpy as np

from . import Sim

PARAMS = ("alpha", "phi_g", "B")
OUT_COLS = (2, 3, 1, 4, 6)  # drag F_Z, electric F_Z, current, torque T_z, Q


def window_outputs(sim, n_steps):
    """Means over the last n_steps history rows of the five outputs."""
    h = sim.history()[-n_steps:]
    return h[:, OUT_COLS].mean(axis=0)


def _run(cfg, states, n_steps, mode, tape=None):
    s = Sim(cfg)
    for sp, st in enumerate(states):
        if st is not None and len(st):
            s.add_particles(sp, st)
    if tape is not None:
        s.set_tape(tape)
    s.tape_mode(mode)
    s.step(n_steps)
    if mode == Sim.TAPE_REPLAY and not s.tape_ok():
        raise RuntimeError("replay ran past the end of its decision tape")
    return s


def window_sensitivity(cfg, states, n_steps, h=None):
    """Window means (5,) and their central-difference derivatives (5, 3)
    along (alpha, phi_g, B) with the decisions of the unperturbed run."""
    h = {**dict(alpha=1e-6, phi_g=1e-6, B=1e-6), **(h or {})}
    base = _run(cfg, states, n_steps, Sim.TAPE_RECORD)
    tape = base.tape()
    vals = window_outputs(base, n_steps)
    jac = np.zeros((len(OUT_COLS), len(PARAMS)))
    for p, key in enumerate(PARAMS):
        out = []
        for sgn in (1.0, -1.0):
            c = dict(cfg)
            c[key] = float(cfg[key]) + sgn * h[key]
            out.append(window_outputs(_run(c, states, n_steps, Sim.TAPE_REPLAY, tape), n_steps))
        jac[:, p] = (out[0] - out[1]) / (2.0 * h[key])
    return vals, jac, tape
