"""Build the CUDA library (liblbm13.so) for sm_103a, in-tree.

The translation units compile in parallel with nvcc and link into
paper_1401_0188_gb300/_build/liblbm13.so, which the ctypes binding loads.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "liblbm13.so")
# bounds-checked build (LBM13_DEBUG): every population access of the step
# kernels is checked and counted (lbm13_debug_violations)
DEBUG_OUT = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_OUT, "liblbm13_debug.so")
SOURCES = ["lbm13_step.cu", "lbm13_step2.cu", "lbm13_batch.cu", "lbm13_multi.cu", "lbm13_aux.cu", "lbm13_api.cu", "lbm13_noalloc.cu", "lbm13_linear.cu", "lbm13_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(home, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "lbm13.h"))
    return files


def build(force=False, verbose=False, extra=(), debug=False):
    out, lib = (DEBUG_OUT, DEBUG_LIB) if debug else (OUT, LIB)
    if debug:
        extra = (*extra, "-DLBM13_DEBUG")
    os.makedirs(out, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in _deps())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest and (debug or not extra):
        return lib
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
