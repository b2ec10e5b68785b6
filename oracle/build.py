"""Build the FP64 CPU oracle (test infrastructure, not part of the product).

Compiles oracle/cacl_oracle.cpp into oracle/libcacl_oracle.so with g++ and
OpenMP. No fast-math: the FP32 comparison form of the wall normal relies on
correctly rounded IEEE division and square root.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cacl_oracle.cpp")
OUT = os.path.join(HERE, "libcacl_oracle.so")


def build(force: bool = False) -> str:
    deps = [SRC, os.path.join(HERE, "cacl_oracle.h")]
    if (not force and os.path.exists(OUT)
            and os.path.getmtime(OUT) >= max(os.path.getmtime(d) for d in deps)):
        return OUT
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", OUT + ".tmp", SRC]
    subprocess.check_call(cmd)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
