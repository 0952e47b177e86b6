"""Build step for the CPU oracle (test infrastructure only).

Compiles ``tp_oracle.c`` with gcc into ``oracle/_build/libtporacle.so``.
Multiply-add contraction is disabled (``-ffp-contract=off``) so that every
binary64 operation rounds exactly as written in the C source, on x86-64 and
on aarch64 alike.  OpenMP is used when the compiler provides it (it only
parallelises the dedispersion loop over DM rows; results do not depend on it).
"""
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "tp_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtporacle.so")

BASE_FLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _stale():
    return (not os.path.exists(LIB)) or os.path.getmtime(LIB) < os.path.getmtime(SRC)


def build(force=False):
    """Compile the oracle if needed and return the path of the shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=OUT_DIR)
    os.close(fd)
    last = None
    for extra in (["-fopenmp"], []):
        cmd = ["gcc", *BASE_FLAGS, *extra, SRC, "-o", tmp, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, LIB)
            return LIB
        last = r.stderr
    os.unlink(tmp)
    raise RuntimeError("oracle build failed:\n" + (last or ""))


if __name__ == "__main__":
    print(build(force=True))
