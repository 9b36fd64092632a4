"""Compile the C oracle into ``oracle/_build/libecho_oracle.so``.

Test infrastructure only.  gcc, FP64, no FMA contraction (``-ffp-contract=off``)
so every product in the oracle is rounded exactly as written.  OpenMP is used
when the compiler supports it; the arithmetic of every cell is the same either
way (reductions are done serially).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "echo_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libecho_oracle.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Build the oracle library if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", SRC, "-o", tmp, "-lm"]
    cmd = base[:1] + ["-fopenmp"] + base[1:]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        # no OpenMP runtime: build single-threaded
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    if verbose:
        sys.stdout.write(r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
