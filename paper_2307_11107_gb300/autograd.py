"""torch.autograd binding of the sensitivity window (apic_sensitivity).

`AdjointWindow.apply(params, cfgs, states, n_steps, precision)` maps the
parameters (alpha, phi_g, B) of every instance, a tensor [instances, 3], to
the window means [instances, 5] of (drag F_Z, electric F_Z, current, torque
T_z, grain charge Q) over n_steps steps from the given particle states; its
backward pass is the vector-Jacobian product with the window's frozen-decision
Jacobian (the derivative apic_adjoint returns), computed in the same forward
run.  The window itself runs in the library's kernels.
"""
import numpy as np
import torch

from .sim import Sim


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
        run = [dict(c, alpha=float(a), phi_g=float(g), B=float(b)) for c, (a, g, b) in zip(cfgs, p)]
        sim = Sim(run, precision=precision)
        try:
            for k, per_inst in enumerate(states):
                for sp, st in enumerate(per_inst):
                    if st is not None and len(st):
                        sim.add_particles(sp, np.asarray(st, dtype=np.float64), instance=k)
            out = sim.sensitivity(int(n_steps))
        finally:
            sim.close()
        ctx.save_for_backward(torch.as_tensor(out["jacobian"], dtype=torch.float64))
        return torch.as_tensor(out["values"], dtype=params.dtype, device=params.device).reshape(p.shape[0], -1)

    @staticmethod
    def backward(ctx, grad_out):
        (jac,) = ctx.saved_tensors  # [instances, 5, 3]
        g = torch.einsum("io,iop->ip", grad_out.detach().to("cpu", torch.float64), jac)
        return g.to(grad_out.dtype).to(grad_out.device), None, None, None, None
