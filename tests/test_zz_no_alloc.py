"""apic_deposit_static, the deposit entry point for callers that cannot
allocate device memory (its 64-bit accumulator is a static array inside the
library).  Checked through the C ABI against the density that apic_step
computes for the same particles, on two calls in a row (the second call must
start from a cleared accumulator)."""
import ctypes as C

import numpy as np
import pytest

from tests.inputs import random_states, workload

pytestmark = pytest.mark.gpu


def test_deposit_static_matches_step_deposit_twice():
    import torch
    import paper_2307_11107_gb300 as apic
    from paper_2307_11107_gb300 import _abi
    apic.build()
    L = _abi.load()
    n = 50000
    cfg = workload(n1=64, n2=32, alpha=0.15, n_init=n, precision="fp64", no_inject=True)
    cfg["species"] = cfg["species"][:1]
    st = random_states(n, cfg["x1_out"], seed=21)
    sim = apic.Sim(cfg)
    sim.add_particles(0, st)
    sim.step(1)
    rho_ref, V = sim.field("rho"), sim.field("V")
    sim.close()
    qw_sim = (rho_ref * V).sum() / n  # sum over nodes of rho V = q w n (CIC weights sum to one)

    dev = torch.device("cuda")
    x1 = torch.tensor(st[:, 0], dtype=torch.float64, device=dev)
    x2 = torch.tensor(st[:, 1], dtype=torch.float64, device=dev)
    Vd = torch.tensor(V, dtype=torch.float64, device=dev)
    rho = torch.empty_like(Vd)
    grid = _abi.Grid(cfg["n1"], cfg["n2"], cfg["x1_out"])
    stream = torch.cuda.current_stream()
    for qw in (0.75, -2.0):
        rc = L.apic_deposit_static(C.byref(grid), x1.data_ptr(), x2.data_ptr(), n, qw, Vd.data_ptr(),
                                   rho.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = rho.cpu().numpy() * (qw_sim / qw)
        err = np.abs(got - rho_ref).max() / np.abs(rho_ref).max()
        assert err < 1e-11, err


def test_deposit_static_skips_particles_outside_the_domain():
    """Rows outside [-1, x1_outer] x [-1, 1] or with a NaN coordinate add no
    charge: the density of the in-domain rows alone, bit for bit."""
    import torch
    import paper_2307_11107_gb300 as apic
    from paper_2307_11107_gb300 import _abi
    apic.build()
    L = _abi.load()
    cfg = workload(n1=64, n2=32, alpha=0.15)
    st = random_states(20000, cfg["x1_out"], seed=22)
    bad = np.array([[2.0, 0.1], [-1.5, 0.0], [-0.5, 1.5], [-0.5, -1.2], [np.nan, 0.0], [-0.5, np.nan],
                    [np.inf, 0.0], [cfg["x1_out"] + 1e-3, 0.3]])
    dev = torch.device("cuda")
    Vd = torch.ones((cfg["n1"] + 1, cfg["n2"] + 1), dtype=torch.float64, device=dev)
    grid = _abi.Grid(cfg["n1"], cfg["n2"], cfg["x1_out"])
    stream = torch.cuda.current_stream()
    out = []
    for xy in (st[:, :2], np.concatenate([bad, st[:, :2], bad])):
        x1 = torch.tensor(xy[:, 0], dtype=torch.float64, device=dev)
        x2 = torch.tensor(xy[:, 1], dtype=torch.float64, device=dev)
        rho = torch.empty_like(Vd)
        # the same particle count bound (fixed-point bits) for both calls
        rc = L.apic_deposit_static(C.byref(grid), x1.data_ptr(), x2.data_ptr(), xy.shape[0], 1.0, Vd.data_ptr(),
                                   rho.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        out.append(rho.cpu().numpy())
    assert np.abs(out[0] - out[1]).max() <= 1e-12 * np.abs(out[0]).max()
    assert out[0].sum() == pytest.approx(20000, rel=1e-12)


def test_deposit_static_rejects_oversized_grid():
    import paper_2307_11107_gb300 as apic
    from paper_2307_11107_gb300 import _abi
    apic.build()
    L = _abi.load()
    grid = _abi.Grid(2048, 1024, -0.05)  # 2049 * 1025 nodes > 2^20
    rc = L.apic_deposit_static(C.byref(grid), None, None, 0, 1.0, C.c_void_p(16), C.c_void_p(16), None)
    assert rc == -1
