"""Synthetic workloads of the benchmark and the tests (definitions only).

Units as in include/apic.h (R0 = lambda_De, 1/omega_pe, Te/e, n0 = 1).  The
shape parameter is alpha of Eqs. 1-5; the configurations' "a" values are read
as alpha = a / 2 (the coordinates are one-to-one only for |alpha| < 1/4).
Grids are counted in cells.
"""
import numpy as np

ELECTRON = dict(q=-1.0, m=1.0, T=1.0)


def ion(T=1.0, m=1836.0):
    return dict(q=1.0, m=m, T=T)


def spherical_small(precision="fp64"):
    """Spherical grain alpha = 0, B = 0, 64 x 32 cells, x1 in [-1, -0.1],
    phi_g = -2.5, 1e5 macro-particles per species, dt = 0.1, FP64 (200 steps)."""
    return dict(name="sphere_64x32_2e5", alpha=0.0, x1_out=-0.1, phi_g=-2.5, phi_out=0.0, B=0.0, dt=0.1,
                n1=64, n2=32, species=[dict(ELECTRON, n_init=100000), dict(ion(1.0), n_init=100000)],
                seed=1, precision=precision, poisson_tol=1e-13, poisson_max_iter=40, steps=200)


def dipole_256(precision="fp32", n_per_species=10_000_000):
    """Dipole-shaped grain a = 0.3 (alpha = 0.15) with axial B = 1 (electron
    gyroradius = R0), 256 x 128 cells, x1_out = -0.05, Ti = 0.5 Te,
    1e7 macro-particles per species, dt = 0.1 (2000 steps)."""
    return dict(name="dipole_a0.3_256x128_2e7", alpha=0.15, x1_out=-0.05, phi_g=-2.5, phi_out=0.0, B=1.0, dt=0.1,
                n1=256, n2=128, species=[dict(ELECTRON, n_init=n_per_species), dict(ion(0.5), n_init=n_per_species)],
                seed=1, precision=precision, poisson_tol=1e-10, poisson_max_iter=20, sort_interval=8, poisson_guess=1, steps=2000)


def dipole_256_boltzmann(precision="fp32", n_ions=10_000_000):
    """The 256 x 128 dipole with Boltzmann electrons: 1e7 ions only, the
    nonlinear Poisson problem solved by Newton each step, dt = 1.0 (ten times
    the two-species step; the ion plasma period is 43 times the electron one)."""
    c = dipole_256(precision)
    c.update(name="dipole_a0.3_256x128_1e7ions_boltzmann", species=[dict(ion(0.5), n_init=n_ions)], dt=1.0,
             boltzmann=True, poisson_tol=1e-10, poisson_max_iter=30, newton_iters=8, steps=200)
    return c


def dipole_256_floating(precision="fp32", n_per_species=10_000_000):
    """The 256 x 128 dipole with an isolated grain (its potential follows the
    collected charge, starting from -2.5)."""
    c = dipole_256(precision, n_per_species)
    c.update(name="dipole_a0.3_256x128_2e7_floating", floating=True)
    return c


def dipole_1024(precision="fp32", n_per_species=50_000_000):
    """Precision form at scale: a = 0.45 (alpha = 0.225), 1024 x 512 cells,
    5e7 macro-particles per species, FP32 particles, the Poisson problem solved
    in FP32 inside the FP64 residual refinement to 1e-10 (1000 steps)."""
    return dict(name="dipole_a0.45_1024x512_1e8", alpha=0.225, x1_out=-0.05, phi_g=-2.5, phi_out=0.0, B=1.0,
                dt=0.1, n1=1024, n2=512,
                species=[dict(ELECTRON, n_init=n_per_species), dict(ion(0.5), n_init=n_per_species)],
                seed=1, precision=precision, poisson_tol=1e-10, poisson_max_iter=30, sort_interval=8, steps=1000)


def batched_48(seed=2, scale=1.0):
    """48 uneven instances: a in [0, 0.5) (alpha = a/2, capped at 0.24),
    phi_g in [-4, -1], B in {0, 1}, grids 128x64 .. 512x256 (multiples of 32),
    1e5 .. 5e6 macro-particles per species (log-uniform)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(48):
        a = rng.uniform(0.0, 0.5)
        n1 = int(np.exp(rng.uniform(np.log(128), np.log(512))) // 32 * 32)
        npart = int(np.exp(rng.uniform(np.log(1e5), np.log(5e6))) * scale)
        out.append(dict(name="inst%02d" % k, alpha=min(a / 2, 0.24), x1_out=-0.05, phi_g=rng.uniform(-4.0, -1.0),
                        phi_out=0.0, B=float(rng.integers(0, 2)), dt=0.1, n1=n1, n2=n1 // 2,
                        species=[dict(ELECTRON, n_init=npart), dict(ion(0.5), n_init=npart)], seed=2, instance=k,
                        precision="fp32", poisson_tol=1e-8, poisson_max_iter=20, sort_interval=8))
    return out
