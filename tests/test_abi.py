"""The C ABI library: builds for sm_103a, loads, and exports every entry point
declared in include/apic.h; the ctypes mirror has the header's layout.
No GPU work is done here."""
import os
import re
import subprocess
import tempfile

import pytest

import paper_2307_11107_gb300 as apic
from paper_2307_11107_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "apic.h")


def test_library_builds_and_exports_declared_symbols():
    apic.build()
    L = _abi.load()
    declared = set(re.findall(r"^\s*(?:const char\*|int32_t|int)\s+(apic_\w+)\s*\(", open(HDR).read(), re.M))
    assert declared == set(_abi.SYMBOLS), declared ^ set(_abi.SYMBOLS)
    for name in declared:
        assert hasattr(L, name)
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared:
        assert re.search(r"\bT %s\b" % name, out), name


def test_struct_layout_matches_header():
    import ctypes
    src = r'''
    #include <stdio.h>
    #include <stddef.h>
    #include "apic.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(apic_config_t), sizeof(apic_tallies_t), sizeof(apic_species_t),
             offsetof(apic_config_t, seed), offsetof(apic_config_t, poisson_tol), offsetof(apic_tallies_t, step),
             sizeof(apic_stats_t), offsetof(apic_stats_t, sort_ms));
      return 0;
    }'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(td, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = list(map(int, subprocess.check_output([exe]).split()))
    exp = [ctypes.sizeof(_abi.Config), ctypes.sizeof(_abi.Tallies), ctypes.sizeof(_abi.Species),
           _abi.Config.seed.offset, _abi.Config.poisson_tol.offset, _abi.Tallies.step.offset,
           ctypes.sizeof(_abi.Stats), _abi.Stats.sort_ms.offset]
    assert vals == exp


def test_invalid_configs_rejected_without_gpu_work():
    """Argument validation happens before any device call."""
    import ctypes as C
    from tests.inputs import workload
    L = _abi.load()
    for bad, code in ((dict(alpha=0.3), -2), (dict(x1_out=-1.5), -2), (dict(n2=4), -1)):
        cfg = apic.make_config(dict(workload(), **bad), "fp64")
        h = C.c_void_p()
        assert L.apic_create(C.byref(cfg), None, None, C.byref(h)) == code
        assert not h.value


def test_null_arguments():
    import ctypes as C
    L = _abi.load()
    assert L.apic_create(None, None, None, None) == -1
    assert L.apic_destroy(None) == 0
    assert L.apic_step(None, 1) == -1
    assert L.apic_set_schedule(None, 0, 0, 0, 0) == -1
    assert L.apic_checkpoint_size(None, None) == -1
    assert L.apic_checkpoint_save(None, None, 0) == -1
    assert L.apic_checkpoint_load(None, None, 0) == -1
    assert L.apic_last_error(None) == b"null simulation"
