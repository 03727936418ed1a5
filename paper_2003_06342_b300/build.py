"""Build the CUDA library liblbmpf.so in-tree for sm_103a (B300).

nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3, one shared
object from csrc/*.cu, linked against the shared CUDA runtime (the one the
PyTorch process has already loaded).  `python paper_2003_06342_b300/build.py`
rebuilds it (run it as a script: importing the package would load the old
library first).

A second object, liblbmpf_debug.so, is the same sources compiled with
-DLBM_CHECK_BOUNDS: every population and field index a kernel computes is
checked against its buffer before the access, a failing access is skipped and
recorded, and lbm_sync reports LBM_EBOUNDS.  The binding loads it instead of
the release library when LBM_PF_DEBUG=1 is set in the environment.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbmpf.so")
LIB_DEBUG = os.path.join(LIBDIR, "liblbmpf_debug.so")
SOURCES = ["api.cu", "lbm2d.cu", "lbm3d.cu", "reduce.cu", "noalloc.cu", "adjoint2d.cu", "lbm2d_tma.cu",
           "lbm3d_tma.cu", "cac2d.cu", "cac3d.cu", "health.cu", "columns.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _run(cmd, what, verbose):
    res = subprocess.run(cmd, cwd=CSRC, capture_output=True, text=True)
    if verbose or res.returncode != 0:
        sys.stdout.write(res.stdout)
        sys.stderr.write(res.stderr)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed building {what}")


def _jobs(out, defines, ptxas_info):
    """(compile commands, objects) of one library: one object per source."""
    tag = os.path.splitext(os.path.basename(out))[0]
    objdir = os.path.join(HERE, "_build", tag)
    os.makedirs(objdir, exist_ok=True)
    flags = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *defines]
    if ptxas_info:
        flags.insert(0, "-Xptxas=-v")
    objs = [os.path.join(objdir, os.path.splitext(s)[0] + ".o") for s in SOURCES]
    jobs = [([nvcc(), *flags, "-c", os.path.join(CSRC, s), "-o", o], s) for s, o in zip(SOURCES, objs)]
    return jobs, objs


def build(verbose=False, ptxas_info=False, debug=True):
    """Build the release library (and, unless debug=False, the bounds-checking
    one): every object compiled in parallel, then one shared link per
    library.  Returns the release library's path."""
    os.makedirs(LIBDIR, exist_ok=True)
    libs = [(LIB, [], ptxas_info)] + ([(LIB_DEBUG, ["-DLBM_CHECK_BOUNDS"], False)] if debug else [])
    plan = [(out,) + _jobs(out, defines, pi) for out, defines, pi in libs]
    jobs = [j for _, js, _ in plan for j in js]
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for f in [ex.submit(_run, cmd, what, verbose) for cmd, what in jobs]:
            f.result()
    for out, _, objs in plan:
        _run([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
              "-o", out, *objs], os.path.basename(out), verbose)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv, debug="--no-debug" not in sys.argv)
    print(LIB)
