"""Compile the CPU oracle into oracle/_build/liboracle.so.

TEST INFRASTRUCTURE ONLY: the oracle is the reference the CUDA path is checked
against; nothing in the product path loads it.
"""
import fcntl
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["basis.cpp", "dgfv_oracle.cpp"]
HEADERS = ["basis.hpp", "physics.hpp", "scalar_types.hpp", "dgfv_oracle.h"]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in SOURCES + HEADERS + ["build.py"])


def build(force: bool = False) -> str:
    """Build the oracle library if it is missing or older than its sources
    (concurrent callers serialise on a lock file)."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    with open(os.path.join(OUT_DIR, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not _stale():
                return LIB
            tmp = LIB + f".tmp{os.getpid()}"
            # -ffp-contract=off: no fused multiply-add contraction, so x86 and Arm
            # hosts round identically.
            cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                   "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
            subprocess.run(cmd, check=True)
            os.replace(tmp, LIB)
            return LIB
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
