"""Build libapic.so (sm_103a) in-tree with nvcc.

Translation units (compiled in parallel):
  particles.cu  twice: FP64 particles (-fmad=false, the parity build) and FP32
  poisson.cu    twice: FP64 and FP32 multigrid preconditioner
  fields.cu     node fields and bookkeeping, the isolated grain's correction and
                the Newton linearisation of Boltzmann electrons (FP64, -fmad=false)
  bcr.cu        block cyclic reduction solve (FP32 blocks, FP64 refinement)
  apic.cu       host set-up and the C ABI
  tangent.cu    twice: the sensitivity window's particle kernels in FP64
                (-fmad=false, with its node kernels) and FP32
  deposit_static.cu  the deposit entry point that uses no caller-side allocation
  probe.cu      the FP32 fused-multiply-add throughput probe (the ALU ceiling)
  nd_factor.cpp the host nested-dissection factorisation of the Poisson system
  adjoint.cu    twice: the reverse sweep of the sensitivity window in FP64 (-fmad=false,
                with its node kernels) and FP32
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libapic.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
BASE = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math",
        "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]

UNITS = [
    ("particles.cu", "particles_f64.o", ["-DAPIC_REAL=double", "-fmad=false"]),
    ("particles.cu", "particles_f32.o", ["-DAPIC_REAL=float", "--use_fast_math"]),
    ("poisson.cu", "poisson_f64.o", ["-DAPIC_POISSON_REAL=double", "-DAPIC_POISSON_COMMON=1"]),
    ("poisson.cu", "poisson_f32.o", ["-DAPIC_POISSON_REAL=float", "-DAPIC_POISSON_COMMON=0"]),
    ("fields.cu", "fields.o", ["-fmad=false"]),
    ("bcr.cu", "bcr.o", []),
    ("apic.cu", "apic.o", []),
    ("tangent.cu", "tangent_f64.o", ["-DAPIC_REAL=double", "-DAPIC_TANGENT_COMMON", "-fmad=false"]),
    ("tangent.cu", "tangent_f32.o", ["-DAPIC_REAL=float"]),
    ("deposit_static.cu", "deposit_static.o", ["-fmad=false"]),
    ("probe.cu", "probe.o", []),
    ("nd_factor.cpp", "nd_factor.o", []),
    ("adjoint.cu", "adjoint_f64.o", ["-DAPIC_REAL=double", "-DAPIC_ADJOINT_COMMON", "-fmad=false"]),
    ("adjoint.cu", "adjoint_f32.o", ["-DAPIC_REAL=float"]),
]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "apic.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False, extra=()):
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_unit(u):
        src, obj, flags = u
        cmd = [nvcc()] + ARCH + BASE + list(flags) + list(extra) + ["-c", os.path.join(CSRC, src), "-o",
                                                                    os.path.join(BUILD, obj)]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return r.stderr

    with ThreadPoolExecutor(max_workers=min(6, os.cpu_count() or 1)) as ex:
        logs = list(ex.map(compile_unit, UNITS))
    if verbose:
        for l in logs:
            if l.strip():
                print(l)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [os.path.join(BUILD, u[1]) for u in UNITS]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
