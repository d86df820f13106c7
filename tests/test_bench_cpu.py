"""The benchmark's reference arm (the FP64 oracle on a bounded sample of the
bench workload, on the host cores) prints one JSON line with the keys the
measurement contract asks for; it needs no GPU.  The oracle's all-core leg
(independent replicas in spawned processes) and the reference arm's grid
choice are checked on small cases."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    # the 256 x 128 workload keeps the oracle's set-up short here; the default
    # (1024 x 512) runs the same code on the grid reference_grid picks
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "dipole256",
                          "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "particle-steps/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["cpu"]
    assert d["config"]["workload"] == "dipole_a0.3_256x128_2e7"
    assert d["config"]["oracle_grid_cells"] == [256, 128]


def test_reference_grid_fits_budget():
    """Short runs keep the workload's own grid; long ones halve it until the
    oracle's factorisation and solves fit the budget."""
    c = bench.workload(None, "dipole1024")
    assert bench.reference_grid(c, 25) == (1024, 512)
    n1, n2 = bench.reference_grid(c, 1030)
    assert (n1, n2) in ((512, 256), (256, 128)) and n1 == 2 * n2


def test_all_core_replicas():
    """Two spawned replicas of a small sample advance twice the particles of
    one, in about the same time."""
    c = bench.workload(None, "dipole256")
    v1, s1 = bench.run_oracle(c, 5000, 3, 1, 1, grid=(64, 32))
    v2, s2 = bench.run_oracle(c, 5000, 3, 1, 2, grid=(64, 32))
    assert v1 > 0 and v2 > 0 and s1 > 0 and s2 > 0
