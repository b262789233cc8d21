"""Build libblindmatch.so (the CUDA library behind include/blindmatch.h) in-tree.

Compiles each translation unit of csrc/ for sm_103a in parallel with nvcc and
links them into paper_2408_06167_gb300/_build/libblindmatch.so.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libblindmatch.so")
SOURCES = ["api.cu", "kernels.cu", "ks_fused.cu", "server.cu", "host.cpp", "profile.cpp", "noalloc.cu", "tune.cu", "encrypt.cu"]
HEADERS = ["bm_internal.h", "bm_math.cuh", "ntt_reg.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp", "-Xcompiler", "-D_GLIBCXX_ASSERTIONS",
            "-I", os.path.join(ROOT, "include"), "-I", SRC] + ARCH


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "blindmatch.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [NVCC] + _flags() + ["-c", os.path.join(SRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd = [NVCC, "-x", "cu"] + cmd[1:]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile (if sources changed) and return the path of libblindmatch.so."""
    os.makedirs(OUT, exist_ok=True)
    if not force and not _stale():
        return LIB
    with concurrent.futures.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-fopenmp", "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
