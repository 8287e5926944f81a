"""Build the CPU oracle (test infrastructure) as a shared library.

The oracle is plain C++17, single-threaded, compiled with contraction and
fast-math off so that every fp32 operation is the one written in the source.
Only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gpz_oracle.cpp")
LIB = os.path.join(HERE, "libgpz_oracle.so")

CXXFLAGS = ["-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile oracle/libgpz_oracle.so if it is missing or older than its sources.

    GPZ_ORACLE_LIB names another build of the oracle to load instead; the
    mutation test uses it to run the pins against copies with planted
    mistakes."""
    override = os.environ.get("GPZ_ORACLE_LIB")
    if override:
        return override
    deps = [SRC, os.path.join(HERE, "gpz_oracle.h"), os.path.abspath(__file__)]
    if not force and os.path.exists(LIB):
        if os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in deps):
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++"] + CXXFLAGS + [SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
