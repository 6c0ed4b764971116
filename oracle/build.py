"""Build the CPU oracle (test infrastructure only) into oracle/liboracle.so
(dg_oracle.cpp: Cartesian operator, dg_curved.cpp: curvilinear operator).

Plain g++ with OpenMP; -ffp-contract=off keeps every multiply and add separately rounded
except where the oracle calls fma() itself.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dg_oracle.cpp")
SRC2 = os.path.join(HERE, "dg_curved.cpp")
LIB = os.path.join(HERE, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    hdr = os.path.join(HERE, "dg_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(SRC2), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", SRC, SRC2, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
