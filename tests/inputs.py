"""Seeded synthetic inputs shared by the oracle and the CUDA path in the tests.

This module holds no arithmetic of the method: it only draws random numbers
(numpy, seeded) and builds workload dictionaries.  Both sides receive exactly
the same arrays.
"""
import numpy as np

ELECTRON = dict(q=-1.0, m=1.0, T=1.0)
ION = dict(q=1.0, m=1836.0, T=1.0)


def workload(n1=64, n2=32, alpha=0.0, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, B=0.0, dt=0.1,
             n_init=100000, Ti=1.0, seed=1, **kw):
    d = dict(alpha=alpha, x1_out=x1_out, phi_g=phi_g, phi_out=phi_out, B=B, dt=dt, n1=n1, n2=n2,
             species=[dict(ELECTRON, n_init=n_init), dict(ION, T=Ti, n_init=n_init)], seed=seed)
    d.update(kw)
    return d


def random_states(n, x1_out, seed, vscale=1.0, margin=1e-3):
    """n rows of (x1, x2, vR, vZ, vTheta): logical positions uniform inside the
    box (x1 in (-1, x1_out), x2 in (-1, 1)), velocities standard normal."""
    rng = np.random.default_rng(seed)
    x1 = rng.uniform(-1.0 + margin, x1_out - margin, n)
    x2 = rng.uniform(-1.0 + margin, 1.0 - margin, n)
    v = rng.standard_normal((n, 3)) * vscale
    return np.column_stack([x1, x2, v]).astype(np.float64)


def random_rho(n1, n2, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n1 + 1, n2 + 1)) * scale
