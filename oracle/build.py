"""Compile the C oracle into oracle/_build/libljoracle.so and the CPU Verlet-list baseline into
oracle/_build/libcellverlet.so (gcc, FP64, no FMA contraction, OpenMP when available)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "ljoracle.c")
LIB = os.path.join(OUT_DIR, "libljoracle.so")
CV_SRC = os.path.join(HERE, "cellverlet.c")
CV_LIB = os.path.join(OUT_DIR, "libcellverlet.so")


def _compile(src: str, lib: str, force: bool) -> str:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = lib + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        # no OpenMP runtime: still correct, just single-threaded
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Build the oracle library if missing or older than its source; return its path."""
    return _compile(SRC, LIB, force)


def build_cellverlet(force: bool = False) -> str:
    """Build the CPU Verlet-list baseline if missing or older than its source; return its path."""
    return _compile(CV_SRC, CV_LIB, force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_cellverlet(force=True))
