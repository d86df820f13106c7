"""Sensitivity window (forward-mode derivatives along alpha, phi_g, B) of the
CUDA path against the oracle's frozen-decision central differences, and
against the closed forms of the vacuum sphere."""
import numpy as np
import pytest

from oracle.sensitivity import window_sensitivity
from tests.inputs import random_states, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import paper_2307_11107_gb300 as apic
    apic.build()
    return apic


def _states(n, x1_out, seed):
    return [random_states(n, x1_out, seed=seed), random_states(n, x1_out, seed=seed + 1, vscale=0.03)]


def _gpu_window(apic, cfg, states, K, precision):
    s = apic.Sim(cfg, precision=precision)
    for sp, st in enumerate(states):
        if st is not None:
            s.add_particles(sp, st)
    out = s.sensitivity(K)
    return s, out["values"][0], out["jacobian"][0]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vacuum_sphere(apic, precision):
    """No particles, alpha = 0: Q = 4 pi (phi_g - phi_out)/(1 + x1_out) exactly
    on the grid, dQ/dphi_g = 4 pi/(1 + x1_out); mirror symmetry gives
    dQ/dalpha = 0 and F_Z = dF_Z/dphi_g = 0; B acts on particles only."""
    cfg = workload(n1=64, n2=32, alpha=0.0, n_init=1000, no_inject=True, poisson_tol=1e-12, poisson_max_iter=60)
    _, v, J = _gpu_window(apic, cfg, [None, None], 3, precision)
    x1o = cfg["x1_out"]
    assert v[4] == pytest.approx(4 * np.pi * (cfg["phi_g"] - cfg["phi_out"]) / (1 + x1o), rel=1e-9)
    assert J[4, 1] == pytest.approx(4 * np.pi / (1 + x1o), rel=1e-9)
    assert abs(J[4, 0]) < 1e-8 * abs(v[4])
    assert abs(v[1]) < 1e-8 and abs(J[1, 1]) < 1e-8
    assert np.all(J[[0, 2, 3]] == 0.0) and np.all(J[:, 2] == 0.0)


@pytest.mark.parametrize("precision,alpha,B,fe", [("fp64", 0.15, 0.5, False), ("fp64", -0.2, 1.0, False),
                                                  ("fp32", 0.15, 0.5, False), ("fp64", 0.15, 0.5, True)])
def test_window_against_oracle_differences(apic, precision, alpha, B, fe):
    """Window means and the 5 x 3 Jacobian against the oracle's central
    differences with the decisions of its unperturbed run (also with the
    conservative operator, whose alpha derivative includes the node volumes')."""
    n, K = 4000, 5
    cfg = workload(n1=32, n2=16, alpha=alpha, B=B, n_init=n, x1_out=-0.1, seed=3, poisson_tol=1e-13,
                   poisson_max_iter=80, fe_operator=fe)
    st = _states(n, cfg["x1_out"], 31)
    if precision == "fp32":
        st = [s.astype(np.float32).astype(np.float64) for s in st]
    vo, Jo, _ = window_sensitivity(cfg, st, K)
    s, vg, Jg = _gpu_window(apic, cfg, st, K, precision)
    vscale = np.abs(vo) + 1e-12
    scale = np.abs(Jo).max(axis=1, keepdims=True) + 1e-30
    ev = np.abs(vg - vo) / vscale
    eJ = np.abs(Jg - Jo) / scale
    print(f"\n{precision} alpha={alpha} B={B}: values rel err {ev.max():.2e}, jacobian rel err (row scale) "
          f"{eJ.max():.2e}\n oracle J =\n{Jo}\n gpu J =\n{Jg}")
    # Row 2 (current) is q w (events) / dt under frozen decisions: its only
    # entry, I d ln w / d alpha (~1e-5 relative), is below the rounding of the
    # differences, so it is checked against d ln V_dom / d alpha instead.
    rows = [0, 1, 3, 4]
    if precision == "fp64":
        assert ev.max() < 1e-9
        assert eJ[rows].max() < 1e-6
    else:
        assert ev.max() < 1e-4
        assert eJ[rows].max() < 1e-3
    assert Jg[2, 1] == 0.0 and Jg[2, 2] == 0.0
    import oracle
    h = 1e-4
    vp = oracle.Sim(dict(cfg, alpha=alpha + h)).scalars()["V_dom"]
    vm = oracle.Sim(dict(cfg, alpha=alpha - h)).scalars()["V_dom"]
    assert Jg[2, 0] == pytest.approx(vg[2] * (np.log(vp) - np.log(vm)) / (2 * h), rel=1e-5)
    # the window advanced the simulation; stepping on is still valid
    s.step(2)
    assert s.tallies()["step"] == K + 2


@pytest.mark.slow
def test_adjoint_form_configuration_against_oracle_differences(apic):
    """The adjoint form's configuration: alpha = 0.15 (a = 0.3), B = 1,
    256 x 128 cells, 1e6 particles per species, a window of K = 10 steps with
    injection.  The oracle's central differences replay every decision of its
    unperturbed run, each particle's cell included, so they converge at
    O(h^2) to the frozen-decision derivative.  FP64 tangents: all rows but the
    current (whose differences are rounding-limited; checked above) within
    1e-3 of each row's scale, against differences at h = 1e-5 for every
    column and at the configuration's h = 1e-4 for phi_g and B (at 1e-4 the
    alpha column still carries an O(h^2) error of up to 10 %: the geometry's
    second derivatives are large).  FP32 tangents: an FP32 trajectory holds
    other cells than the FP64 one for some 1e4 particle-steps, and each such
    particle's derivative moves by the jump of the bilinear weights' slope,
    so only the rows that no field derivative dominates, drag and torque, are
    held to the FP64 derivative (within 5e-3)."""
    n, K = 1_000_000, 10
    cfg = workload(n1=256, n2=128, alpha=0.15, B=1.0, x1_out=-0.05, n_init=n, Ti=0.5, seed=5,
                   poisson_tol=1e-12, poisson_max_iter=60)
    st = [random_states(n, cfg["x1_out"], seed=71), random_states(n, cfg["x1_out"], seed=72, vscale=0.0165)]
    st = [x.astype(np.float32).astype(np.float64) for x in st]
    vo, J5, _ = window_sensitivity(cfg, st, K, h=dict(alpha=1e-5, phi_g=1e-5, B=1e-5))
    _, J4, _ = window_sensitivity(cfg, st, K, h=dict(alpha=1e-5, phi_g=1e-4, B=1e-4))
    rows = [0, 1, 3, 4]
    scale = np.abs(J5).max(axis=1, keepdims=True) + 1e-30
    _, vg, Jg = _gpu_window(apic, cfg, st, K, "fp64")
    e5 = (np.abs(Jg - J5) / scale)[rows]
    e4 = (np.abs(Jg - J4) / scale)[rows][:, 1:]
    ev = np.abs(vg - vo) / (np.abs(vo) + 1e-12)
    _, vf, Jf = _gpu_window(apic, cfg, st, K, "fp32")
    ef = (np.abs(Jf - Jg) / (np.abs(Jg).max(axis=1, keepdims=True) + 1e-30))[[0, 3]]
    print(f"\nadjoint-form configuration: values {ev.max():.2e}, fp64 vs h=1e-5 {e5.max():.2e}, vs h=1e-4 "
          f"(phi_g, B) {e4.max():.2e}, fp32 drag/torque vs fp64 {ef.max():.2e}\n oracle J (h=1e-5) =\n{J5}"
          f"\n gpu fp64 J =\n{Jg}\n gpu fp32 J =\n{Jf}")
    assert ev.max() < 1e-9
    assert e5.max() < 1e-3 and e4.max() < 1e-3
    assert ef.max() < 5e-3
    # the reverse sweep, one output row at a time, gives the same rows
    Jr = np.zeros_like(Jg)
    for o in range(5):
        s = apic.Sim(cfg, precision="fp64")
        for sp in (0, 1):
            s.add_particles(sp, st[sp])
        Jr[o] = s.adjoint(K, np.eye(5)[o])[0]
        s.close()
    er = (np.abs(Jr - J5) / scale)[rows]
    print(f"reverse sweep vs h=1e-5 differences {er.max():.2e}\n gpu reverse J =\n{Jr}")
    assert er.max() < 1e-3
    assert np.all(np.abs(Jr - Jg)[rows] <= 1e-8 * scale[rows])


@pytest.mark.parametrize("n1,n2,n,K,alpha,B", [(32, 16, 3000, 4, 0.1, 0.7), (64, 32, 60000, 5, -0.2, 1.0)])
def test_reverse_sweep_is_the_transpose_of_the_forward_jacobian(apic, n1, n2, n, K, alpha, B):
    """The reverse sweep (per-step checkpoints, transposed push, gather,
    gradients, Poisson solve and deposit) and the forward tangents
    differentiate the same frozen-decision window: for random output weights
    w and parameter directions v, <w, J v> from the forward Jacobian equals
    <J^T w, v> from the reverse sweep, and J^T w equals w^T J, to rounding
    (FP64); the window means agree too."""
    cfg = workload(n1=n1, n2=n2, alpha=alpha, B=B, n_init=n, seed=5, poisson_tol=1e-13, poisson_max_iter=80)
    st = _states(n, cfg["x1_out"], 51)
    vf, J = _gpu_window(apic, cfg, st, K, "fp64")[1:]
    rng = np.random.default_rng(3)
    for _ in range(2):
        w = rng.standard_normal(5)
        v = rng.standard_normal(3)
        s = apic.Sim(cfg, precision="fp64")
        for sp in (0, 1):
            s.add_particles(sp, st[sp])
        g, vr = s.adjoint(K, w, values=True)
        s.close()
        g, vr = g[0], vr[0]
        lhs, rhs = w @ (J @ v), g @ v
        scale = np.abs(w[:, None] * J * v[None, :]).sum() + 1e-300
        print(f"\n<w, J v> = {lhs:.12e}  <J^T w, v> = {rhs:.12e}")
        assert abs(lhs - rhs) <= 1e-10 * scale
        gs = np.abs(w[:, None] * J).sum(axis=0) + 1e-300
        assert np.all(np.abs(g - w @ J) <= 1e-10 * gs), (g, w @ J)
        assert np.allclose(vr, vf, rtol=1e-12, atol=1e-14)


def test_reverse_sweep_fp32(apic):
    """The FP32 window: reverse sweep and forward tangents agree to FP32
    accuracy (both derivatives of the same FP32 run)."""
    n, K = 20000, 4
    cfg = workload(n1=64, n2=32, alpha=0.15, B=0.5, n_init=n, seed=6, poisson_tol=1e-11, poisson_max_iter=60)
    st = [x.astype(np.float32).astype(np.float64) for x in _states(n, cfg["x1_out"], 61)]
    _, _, J = _gpu_window(apic, cfg, st, K, "fp32")
    w = np.array([0.3, -1.0, 2.0, 0.5, 1e-3])
    s = apic.Sim(cfg, precision="fp32")
    for sp in (0, 1):
        s.add_particles(sp, st[sp])
    g = s.adjoint(K, w)[0]
    s.close()
    gs = np.abs(w[:, None] * J).sum(axis=0) + 1e-300
    assert np.all(np.abs(g - w @ J) <= 1e-4 * gs), (g, w @ J)


def test_batched_window_equals_single(apic):
    """Two instances with different (alpha, phi_g, B) in one batch give the
    values and Jacobians of their single-instance runs."""
    n, K = 3000, 4
    cfgs = [workload(n1=32, n2=16, alpha=0.12, B=0.5, n_init=n, seed=7, poisson_tol=1e-13, poisson_max_iter=80),
            workload(n1=32, n2=16, alpha=-0.1, B=1.0, phi_g=-3.0, n_init=n, seed=7, instance=1,
                     poisson_tol=1e-13, poisson_max_iter=80)]
    sts = [_states(n, c["x1_out"], 61 + 2 * k) for k, c in enumerate(cfgs)]
    b = apic.Sim(cfgs, precision="fp64")
    for k in range(2):
        for sp in (0, 1):
            b.add_particles(sp, sts[k][sp], instance=k)
    out = b.sensitivity(K)
    for k in range(2):
        _, v, J = _gpu_window(apic, cfgs[k], sts[k], K, "fp64")
        assert np.allclose(out["values"][k], v, rtol=1e-10, atol=1e-12)
        scale = np.abs(J).max(axis=1, keepdims=True) + 1e-30
        assert (np.abs(out["jacobian"][k] - J) / scale).max() < 1e-8


def test_autograd_window(apic):
    """apic.AdjointWindow as a torch.autograd.Function (backward: the reverse
    sweep through apic_adjoint_window): on the vacuum sphere the gradient of
    the grain charge is dQ/dphi_g = 4 pi/(1 + x1_out) along phi_g and zero
    along B; with particles, backward equals w^T J of the forward tangents for
    the same window."""
    import torch
    cfg = workload(n1=64, n2=32, alpha=0.0, n_init=1000, no_inject=True, poisson_tol=1e-12, poisson_max_iter=60)
    p = torch.tensor([[cfg["alpha"], cfg["phi_g"], cfg["B"]]], dtype=torch.float64, requires_grad=True)
    v = apic.AdjointWindow.apply(p, [cfg], [[None, None]], 3, "fp64")
    v[0, 4].backward()
    x1o = cfg["x1_out"]
    assert p.grad[0, 1].item() == pytest.approx(4 * np.pi / (1 + x1o), rel=1e-9)
    assert p.grad[0, 2].item() == 0.0
    n, K = 4000, 4
    cfg = workload(n1=32, n2=16, alpha=0.15, B=0.5, n_init=n, x1_out=-0.1, seed=3, poisson_tol=1e-13,
                   poisson_max_iter=80)
    st = _states(n, cfg["x1_out"], 31)
    w = np.array([0.3, -1.0, 2.0, 0.5, 1e-3])
    p = torch.tensor([[cfg["alpha"], cfg["phi_g"], cfg["B"]]], dtype=torch.float64, requires_grad=True)
    v = apic.AdjointWindow.apply(p, [cfg], [st], K, "fp64")
    (v[0] * torch.as_tensor(w)).sum().backward()
    _, _, J = _gpu_window(apic, cfg, st, K, "fp64")
    gs = np.abs(w[:, None] * J).sum(axis=0) + 1e-300
    assert np.all(np.abs(p.grad.numpy()[0] - w @ J) <= 1e-10 * gs)
