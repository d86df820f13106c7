"""Compile the FP64 CPU oracle (test infrastructure) into oracle/libapic_oracle.so.

Plain gcc, no FMA contraction (-ffp-contract=off) so the oracle's arithmetic is
exactly the order written in apic_oracle.c on both x86_64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "apic_oracle.c")
LIB = os.path.join(HERE, "libapic_oracle.so")


def build(force: bool = False) -> str:
    hdr = os.path.join(HERE, "apic_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
