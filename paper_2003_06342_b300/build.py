"""Build the CUDA library liblbmpf.so in-tree for sm_103a (B300).

nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3, one shared
object from csrc/*.cu, linked against the shared CUDA runtime (the one the
PyTorch process has already loaded).  `python paper_2003_06342_b300/build.py`
rebuilds it (run it as a script: importing the package would load the old
library first).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "liblbmpf.so")
SOURCES = ["api.cu", "lbm2d.cu", "lbm3d.cu", "reduce.cu", "noalloc.cu", "adjoint2d.cu", "lbm2d_tma.cu",
           "lbm3d_tma.cu", "cac2d.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(verbose=False, ptxas_info=False):
    os.makedirs(LIBDIR, exist_ok=True)
    cmd = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-cudart", "shared", "-Xlinker", "-rpath,/usr/local/cuda/lib64",
           "-o", LIB] + [os.path.join(CSRC, s) for s in SOURCES]
    if ptxas_info:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, cwd=CSRC, capture_output=True, text=True)
    if verbose or res.returncode != 0:
        sys.stdout.write(res.stdout)
        sys.stderr.write(res.stderr)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed building liblbmpf.so")
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
