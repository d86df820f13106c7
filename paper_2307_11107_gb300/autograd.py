"""torch.autograd binding of the window's reverse sweep.

`AdjointWindow.apply(params, cfgs, states, n_steps, precision)` maps the
parameters (alpha, phi_g, B) of every instance, a tensor [instances, 3], to
the window means [instances, 5] of (drag F_Z, electric F_Z, current, torque
T_z, grain charge Q) over n_steps steps from the given particle states.  The
forward pass runs the window's steps (apic_step); the backward pass runs the
window again from the same states through the reverse sweep with per-step
checkpoints (apic_adjoint_window), which returns the gradient of
sum(grad_out * means) at frozen decisions.  All of it runs in the library's
kernels.
"""
import numpy as np
import torch

from .sim import Sim

OUT_COLS = (2, 3, 1, 4, 6)  # history columns of drag F_Z, electric F_Z, current, torque T_z, Q


def _sim(run, states, precision):
    sim = Sim(run, precision=precision)
    for k, per_inst in enumerate(states):
        for sp, st in enumerate(per_inst):
            if st is not None and len(st):
                sim.add_particles(sp, np.asarray(st, dtype=np.float64), instance=k)
    return sim


class AdjointWindow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, cfgs, states, n_steps, precision="fp64"):
        """params: [instances, 3] (alpha, phi_g, B); cfgs: the instances'
        workload dictionaries; states: per instance, per species an array of
        (x1, x2, vR, vZ, vTheta) rows (or None)."""
        p = params.detach().to("cpu", torch.float64).numpy().reshape(-1, 3)
        cfgs = cfgs if isinstance(cfgs, (list, tuple)) else [cfgs]
        if len(cfgs) != p.shape[0]:
            raise ValueError("one parameter row per instance")
        run = [dict(c, alpha=float(a), phi_g=float(g), B=float(b), history_cap=max(int(n_steps) + 1, 16))
               for c, (a, g, b) in zip(cfgs, p)]
        sim = _sim(run, states, precision)
        try:
            sim.step(int(n_steps))
            vals = np.stack([sim.tallies(k)["history"][-int(n_steps):, OUT_COLS].mean(axis=0)
                             for k in range(len(run))])
        finally:
            sim.close()
        ctx.run, ctx.states, ctx.n_steps, ctx.precision = run, states, int(n_steps), precision
        return torch.as_tensor(vals, dtype=params.dtype, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        w = grad_out.detach().to("cpu", torch.float64).numpy()
        sim = _sim(ctx.run, ctx.states, ctx.precision)
        try:
            g = sim.adjoint(ctx.n_steps, w)
        finally:
            sim.close()
        return torch.as_tensor(g, dtype=grad_out.dtype, device=grad_out.device), None, None, None, None
