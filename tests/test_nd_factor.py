"""Host check of the nested-dissection factorisation of the Poisson
correction system (paper_2307_11107_gb300/csrc/nd_factor.cpp): the ordering
covers every unknown once, update sets lie on the enclosing separators, and
the two sweeps the GPU runs (here on the host) solve random operators of the
library's stencil pattern (9 points, pole rows reaching two nodes in x2) to
rounding with the FP64 front matrices and to FP32 accuracy with the stored
FP32 ones, on grids of several shapes and leaf sizes; and the device task
tables, walked as the GPU walks them, give the same solution."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "paper_2307_11107_gb300", "csrc", "nd_factor.cpp")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("nd") / "nd_check")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-o", exe, os.path.join(HERE, "native", "nd_check.cpp"),
                           SRC])
    return exe


@pytest.mark.parametrize("M,N,leaf", [(15, 9, 1), (15, 9, 16), (31, 17, 4), (63, 33, 16), (40, 21, 9),
                                      (127, 65, 16), (7, 65, 16), (255, 9, 4), (255, 129, 16), (511, 257, 16)])
def test_nested_dissection_solves(checker, M, N, leaf):
    out = subprocess.run([checker, str(M), str(N), str(leaf), "7"], capture_output=True, text=True,
                         timeout=300).stdout.split()
    assert out[0] == "OK", out
    r64, r32, tables = float(out[1]), float(out[2]), float(out[-1])
    assert r64 < 1e-12, r64
    assert r32 < 1e-5, r32
    # the GPU's task tables (global offsets of a second instance, row chunks,
    # runs of small fronts) give the host sweep's solution to FP32 rounding
    assert tables < 1e-5, tables
