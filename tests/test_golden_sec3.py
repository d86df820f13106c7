"""The paper's one worked example (Sec. 3) prints only input parameters, no
results (Figs. 1-3 are plots).  These checks derive the dimensionless inputs
from the printed values and confirm the geometry is inside the valid range."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    with open(os.path.join(HERE, "golden", "sec3_example.json")) as f:
        return json.load(f)


def test_sec3_dimensionless_parameters():
    g = _load()
    e, eps0, kB_eV = 1.602176634e-19, 8.8541878128e-12, 1.0
    alpha = g["p_e_m"] / (g["Q_e"] * g["R0_m"])  # Eq. 1: alpha = p / (Q R0)
    assert alpha == pytest.approx(-0.24, rel=1e-12)
    phi0_V = g["Q_e"] * e / (4 * np.pi * eps0 * g["R0_m"])  # Eq. 1: Phi0 = Q / (4 pi eps0 R0)
    assert phi0_V / g["Te_eV"] == pytest.approx(-2.16, abs=0.01)
    lam_D = np.sqrt(eps0 * g["Te_eV"] * kB_eV / (g["n0_m3"] * e))
    assert lam_D / g["R0_m"] == pytest.approx(1.0, abs=0.01)


def test_sec3_geometry_is_valid():
    """|alpha| < 1/4 keeps the x1 = -1 surface a closed grain with a one-to-one
    map (Eqs. 2-5); the oracle accepts alpha = -0.24 and its volumes are positive."""
    s = oracle.Sim(dict(alpha=-0.24, x1_out=-0.1, phi_g=-2.16, phi_out=0, B=0, dt=0.1, n1=32, n2=16,
                        species=[dict(q=-1, m=1, T=1, n_init=1000)], no_field=False))
    assert (s.grid("V") > 0).all()
    with pytest.raises(ValueError):
        oracle.Sim(dict(alpha=0.3, x1_out=-0.1, phi_g=0, phi_out=0, B=0, dt=0.1, n1=8, n2=8,
                        species=[dict(q=-1, m=1, T=1, n_init=10)]))
