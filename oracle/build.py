"""Compile the plain-C oracle (test infrastructure) into oracle/_build/liboracle.so.

Only tests/, __graft_entry__ (build + smoke) and bench.py's cpu_baseline leg use
the oracle.  The library is rebuilt when the C source is newer than the .so.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ckks_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")


def build(force: bool = False, sanitize: bool = False) -> str:
    """sanitize: build with AddressSanitizer and UndefinedBehaviorSanitizer
    (-O1, debug info); Python must then run with both runtimes preloaded:
    LD_PRELOAD="$(gcc -print-file-name=libasan.so) $(gcc -print-file-name=libubsan.so)"
    ASAN_OPTIONS=detect_leaks=0.  Rebuild without it afterwards (force=True)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and not sanitize and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    opt = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer"] if sanitize else ["-O2"]
    cmd = ["gcc"] + opt + ["-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, sanitize="--sanitize" in sys.argv[1:]))
