"""Host check of the fixed-point tally arithmetic (tally_fixed.cuh) used by
the absorption tallies: 128-bit two's-complement sums of signed 64-bit
values, carried through a low and a high word, against Python's exact
integers; and their conversion to FP64 (one rounding, no cancellation for
small negative sums)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("tally") / "tally_fixed_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "native", "tally_fixed_check.cpp")])
    return exe


def _run(exe, values):
    out = subprocess.run([exe], input="\n".join(str(int(v)) for v in values), capture_output=True, text=True,
                         check=True).stdout.split()
    return int(out[0]), int(out[1]), float(out[2])


@pytest.mark.parametrize("case", ["small", "mixed", "huge_pos", "huge_neg", "tiny_negative"])
def test_sum_and_value_exact(checker, case):
    rng = np.random.default_rng(11)
    if case == "small":
        vals = rng.integers(-2 ** 40, 2 ** 40, 5000)
    elif case == "mixed":
        vals = rng.integers(-2 ** 62, 2 ** 62, 5000)
    elif case == "huge_pos":
        vals = rng.integers(2 ** 61, 2 ** 62, 5000)  # the sum passes 2^64: the high word carries
    elif case == "huge_neg":
        vals = -rng.integers(2 ** 61, 2 ** 62, 5000)
    else:
        vals = [-5, 3, -1]  # high word -1, low word near 2^64
    lo, hi, val = _run(checker, vals)
    exact = sum(int(v) for v in vals)
    got = (hi if hi < 2 ** 63 else hi - 2 ** 64) * 2 ** 64 + lo
    assert got == exact
    ref = exact / 2 ** 36
    assert val == pytest.approx(ref, rel=4e-16, abs=0.0)
