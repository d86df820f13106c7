"""Precision form (FP32 particles, the FP32 direct solve (block cyclic
reduction or nested dissection) inside the FP64 residual loop, fixed-point
tallies) against the FP64 oracle.  Single
steps from identical states are compared element by element at FP32
accuracy, also at the sizes where the kernels take their full-size paths;
longer runs, whose trajectories separate (PIC dynamics amplify rounding), are
compared through time-averaged tallies and fields against their statistical
noise."""
import numpy as np
import pytest

import oracle
from tests.inputs import random_states, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apic():
    import paper_2307_11107_gb300 as apic
    apic.build()
    return apic


@pytest.mark.parametrize("alpha,B", [(0.15, 1.0), (-0.24, 0.5)])
def test_fp32_single_step_against_fp64_oracle(apic, alpha, B):
    """One step from the same explicit states: positions and velocities within
    FP32-level error, identical absorbed/escaped sets up to particles within
    rounding of a boundary, rho and phi within FP32 deposit error."""
    n = 40000
    cfg = workload(n1=64, n2=32, alpha=alpha, B=B, n_init=n, precision="fp32", no_inject=True,
                   poisson_tol=1e-12, poisson_max_iter=60)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp, seed, vs in ((0, 31, 1.0), (1, 32, 0.03)):
        st = random_states(n, cfg["x1_out"], seed=seed, vscale=vs)
        st32 = st.astype(np.float32).astype(np.float64)  # both sides start from the FP32 values
        s.add_particles(sp, st32)
        o.add_particles(sp, st32)
    s.step(1)
    o.step(1)
    rho, rho_o = s.field("rho"), o.grid("rho")
    phi, phi_o = s.field("phi"), o.grid("phi")
    # deposit: cell fractions quantised to 16 bits (2^-16 of a cell), positions in FP32
    e_rho = np.abs(rho - rho_o).max() / np.abs(rho_o).max()
    e_phi = np.abs(phi - phi_o).max() / np.abs(phi_o).max()
    print(f"fp32 step alpha={alpha} B={B}: rho {e_rho:.2e} phi {e_phi:.2e}", end="")
    assert e_rho <= 2e-5 and e_phi <= 2e-5
    for sp in (0, 1):
        g, r = s.particles(sp), o.particles(sp)[0]
        assert abs(g.shape[0] - r.shape[0]) <= 2
        if g.shape == r.shape:
            err = np.abs(g - r)
            scale = np.maximum(np.abs(r), np.array([1, 1, 1, 1, 1]) * (1.0 if sp == 0 else 0.03))
            print(f" sp{sp} {(err / scale).max():.2e}", end="")
            assert (err / scale).max() < 2e-4, (err / scale).max(axis=0)
    print()


def _match(g, r, scale):
    """Nearest-neighbour matching of two particle sets (rows x1, x2, vR, vZ,
    vTheta) in scaled coordinates: the matched pairs' largest scaled
    difference, and the rows of either set left without a partner."""
    from scipy.spatial import cKDTree
    tree = cKDTree(r / scale)
    d, k = tree.query(g / scale)
    uniq, cnt = np.unique(k, return_counts=True)
    dup = int((cnt > 1).sum())
    return d, abs(g.shape[0] - r.shape[0]) + dup


@pytest.mark.parametrize("n1,n2,alpha,n", [(256, 128, 0.15, 1_000_000), (64, 512, 0.225, 500_000)])
def test_fp32_step_full_size_paths(apic, n1, n2, alpha, n):
    """One FP32 step at the sizes where the kernels take their full-size
    paths, from the same FP32-rounded states as the FP64 oracle, particles
    sorted by row first (sort interval 8): on 256 x 128 cells the vector
    push's 8-row deposit window is kept across 4096-particle chunks and
    flushed after 15 of them, chunk groups are taken from the counter, fast
    particles deposit outside the window and the Poisson solve is the block
    cyclic reduction (its blocks fit in L2); on 64 x 512 cells the window has
    6 rows of 512 cells and the solve is the nested dissection (the
    reduction's blocks would exceed L2).  rho, phi and every particle are
    compared with the oracle; a second step's density (the push's windowed
    deposit) is compared with the oracle's deposit of the GPU's own positions
    after the first step."""
    cfg = workload(n1=n1, n2=n2, alpha=alpha, B=1.0, x1_out=-0.05, n_init=n, Ti=0.5, precision="fp32",
                   no_inject=True, poisson_tol=1e-12, poisson_max_iter=60, sort_interval=8)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    states = []
    for sp, seed, vs in ((0, 41, 1.0), (1, 42, 0.0165)):
        st = random_states(n, cfg["x1_out"], seed=seed, vscale=vs).astype(np.float32).astype(np.float64)
        s.add_particles(sp, st)
        o.add_particles(sp, st)
        states.append(st)
    s.step(1)
    o.step(1)
    rho, rho_o = s.field("rho"), o.grid("rho")
    phi, phi_o = s.field("phi"), o.grid("phi")
    e_rho = np.abs(rho - rho_o).max() / np.abs(rho_o).max()
    e_phi = np.abs(phi - phi_o).max() / np.abs(phi_o).max()
    print(f"\nfp32 {n1}x{n2} step: rho {e_rho:.2e} phi {e_phi:.2e}", end="")
    assert e_rho <= 2e-5 and e_phi <= 2e-5
    after = []
    for sp, vs in ((0, 1.0), (1, 0.0165)):
        g, r = s.particles(sp), o.particles(sp)[0]
        after.append(g)
        scale = np.array([1.0, 1.0, vs, vs, vs])
        d, unmatched = _match(g, r, scale)
        print(f" sp{sp}: max {d.max():.2e}, unmatched {unmatched}", end="")
        assert unmatched <= 4
        assert np.sort(d)[-unmatched - 1] < 2e-4
    tg, oc = s.tallies()["counts"], o.counts()
    for sp in (0, 1):
        for key in ("absorbed", "escaped"):
            assert abs(tg[sp][key] - oc[sp][key]) <= 4, (sp, key, tg[sp][key], oc[sp][key])
    # the windowed deposit of the push, against the oracle's deposit of the
    # positions the GPU pushed to (16-bit cell fractions against exact ones)
    s.step(1)
    od = oracle.Sim(dict(cfg, no_field=True))
    for sp in (0, 1):
        od.add_particles(sp, after[sp])
    od.deposit()
    rho2, rho2_o = s.field("rho"), od.grid("rho")
    e2 = np.abs(rho2 - rho2_o).max() / np.abs(rho2_o).max()
    print(f" step-2 deposit {e2:.2e}")
    assert e2 <= 2e-5


@pytest.mark.slow
def test_fp32_statistics_against_fp64_oracle(apic):
    """Downsampled dipole run (alpha = 0.15, B = 1, 256 x 128 cells, 1e6
    particles per species, 100 steps): time-averaged currents, drag, grain
    charge and the radial density profile of the FP32-refined GPU run agree
    with the FP64 oracle within their statistical noise."""
    n = 1_000_000
    cfg = workload(n1=256, n2=128, alpha=0.15, B=1.0, x1_out=-0.05, n_init=n, Ti=0.5, seed=7,
                   precision="fp32", poisson_tol=1e-10, poisson_max_iter=40, sort_interval=8)
    s, o = apic.Sim(cfg), oracle.Sim(cfg)
    for sp in (0, 1):
        s.load_volume(sp, n)
        o.load_volume(sp, n)
    steps, avg = 100, 50
    s.step(steps)
    o.step(steps)
    hg, ho = s.tallies()["history"][-avg:], o.history()[-avg:]
    # absorbed events per step are Poisson-distributed: compare the totals
    eg, eo = hg[:, 9].sum(), ho[:, 9].sum()
    assert abs(eg - eo) < 5 * np.sqrt(eg + eo + 1), (eg, eo)
    # grain charge (from phi): the fields average over many particles
    qg, qo = hg[:, 6].mean(), ho[:, 6].mean()
    assert abs(qg - qo) < 0.05 * abs(qo), (qg, qo)
    # resident counts: the runs differ by the noise of the particles lost
    oc = o.counts()
    for col, sp in ((7, 0), (8, 1)):
        a, b = hg[:, col].mean(), ho[:, col].mean()
        churn = oc[sp]["absorbed"] + oc[sp]["escaped"] + oc[sp]["injected"]
        assert abs(a - b) < 5 * np.sqrt(churn + 1), (col, a, b, churn)
    # density per x1 row (volume-weighted mean over x2)
    rho, rho_o, V = s.field("rho"), o.grid("rho"), o.grid("V")
    rg, ro = (rho * V).sum(axis=1), (rho_o * V).sum(axis=1)
    w = o.scalars()["w0"]
    # net charge of a row: ~2 V_row / w macro-particles of charge +-w, two independent runs
    sig = np.sqrt(4 * w * V.sum(axis=1))
    assert (np.abs(rg - ro)[1:-1] < 6 * sig[1:-1]).all(), np.max(np.abs(rg - ro)[1:-1] / sig[1:-1])
    print("fp32 vs fp64 oracle: absorbed", eg, eo, "Q", qg, qo)


def test_vector_push_equals_scalar_push(apic, monkeypatch):
    """The FP32 push that moves four consecutive particles per thread with
    128-bit loads and stores computes what the one-particle push computes:
    the same particles (to FP32 rounding), the same absorbed and escaped
    counts, and densities within one rounding of the 16-bit deposit
    fractions, over several sorted and unsorted steps with injection."""
    runs = []
    for v4 in ("1", "0"):
        monkeypatch.setenv("APIC_PUSH4", v4)
        cfg = workload(n1=128, n2=64, alpha=0.15, B=1.0, x1_out=-0.05, n_init=200_000, Ti=0.5, precision="fp32",
                       seed=9, sort_interval=3)
        s = apic.Sim(cfg)
        for sp in (0, 1):
            s.load_volume(sp, 200_000)
        s.step(4)
        runs.append((s.field("rho"), [s.particles(sp) for sp in (0, 1)], s.tallies()["counts"]))
        s.close()
    (r4, p4, c4), (r1, p1, c1) = runs
    for sp in (0, 1):
        assert c4[sp]["absorbed"] == c1[sp]["absorbed"] and c4[sp]["escaped"] == c1[sp]["escaped"]
        a, b = p4[sp], p1[sp]
        assert a.shape == b.shape
        a, b = a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])]
        assert np.abs(a - b).max() <= 1e-5 * max(1.0, np.abs(b).max())
    assert np.abs(r4 - r1).max() <= 1e-5 * np.abs(r1).max()
