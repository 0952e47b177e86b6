"""Build step of the CUDA library (``libtpdd.so``), sm_103a only.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) and linked into
``paper_1307_5700_gb300/_build/libtpdd.so``.  Floating-point contraction is
off in device code (``--fmad=false``) and in host code
(``-ffp-contract=off``): the delay table, the 8-bit statistics and every
threshold decision are specified operation by operation.

``build(debug=True)`` makes the bounds-checking variant
``paper_1307_5700_gb300/_build_debug/libtpdd_debug.so`` (``-DTP_DEBUG_BOUNDS``):
its kernels check the accesses whose indices come from the plan's geometry,
the delays or the data and record TP_EBOUNDS instead of making them.  The
binding loads it when the environment variable TP_DEBUG_BOUNDS is 1.
"""
import glob
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtpdd.so")
OUT_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(OUT_DIR_DEBUG, "libtpdd_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "--fmad=false", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC]


def nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _inputs():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [
        os.path.abspath(__file__), os.path.join(CSRC, "gen_dispatch.py")]


def stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _inputs())


def generate():
    """Regenerate csrc/dispatch_gen.cuh if its generator is newer."""
    gen = os.path.join(CSRC, "gen_dispatch.py")
    out = os.path.join(CSRC, "dispatch_gen.cuh")
    if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(gen):
        subprocess.run([sys.executable, gen], check=True)


def build(force=False, verbose=False, extra_flags=(), debug=False):
    """Compile and link the library (``debug``: its bounds-checking variant)
    if it is missing or older than its sources; returns the library path."""
    generate()
    out_dir, lib = (OUT_DIR_DEBUG, LIB_DEBUG) if debug else (OUT_DIR, LIB)
    if debug:
        extra_flags = ("-DTP_DEBUG_BOUNDS", *extra_flags)
    if not force and not stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    exe = nvcc()
    objdir = tempfile.mkdtemp(prefix="obj_", dir=out_dir)
    try:
        def compile_one(src):
            obj = os.path.join(objdir, os.path.basename(src) + ".o")
            cmd = [exe, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
            return obj

        # the kernel instantiation units are the slow ones: start them first
        srcs = sorted(sources(), key=lambda f: not os.path.basename(f).startswith("dedisp_p"))
        with ThreadPoolExecutor(max_workers=max(1, min(os.cpu_count() or 8, len(srcs)))) as ex:
            objs = list(ex.map(compile_one, srcs))
        tmp = os.path.join(objdir, os.path.basename(lib))
        cmd = [exe, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
               "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, lib)
    finally:
        shutil.rmtree(objdir, ignore_errors=True)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
