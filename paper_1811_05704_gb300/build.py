"""Build the CUDA library libamg_gb300.so in-tree (sm_103a only).

Each translation unit is compiled in parallel (nvcc for .cu, g++ for the host
setup), then linked into paper_1811_05704_gb300/_build/libamg_gb300.so.  Host
code is compiled with -ffp-contract=off so that the floating-point decisions of
the setup (strength of connection, aggregation ties) are reproducible.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libamg_gb300.so"
LIB_PATH = os.path.join(OUT_DIR, LIB_NAME)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["spmv.cu", "spgemm.cu", "solver.cu", "capi.cu", "noalloc.cu", "tail.cu", "batch.cu", "setup_dev.cu"]
CPP_SOURCES = ["setup_host.cpp", "batch_host.cpp", "server.cpp"]


def _cuda_home():
    return os.environ.get("CUDA_HOME") or os.path.dirname(os.path.dirname(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"))


def _newest_input():
    files = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INCLUDE, "amg.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= _newest_input():
        return LIB_PATH
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    common = ["-O3", "-std=c++17", "-I", INCLUDE]
    jobs = []
    for f in CU_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append([nvcc, *common, *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-c", os.path.join(SRC, f), "-o", obj])
    for f in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, f + ".o")
        jobs.append(["g++", *common, "-fPIC", "-ffp-contract=off", "-I", os.path.join(cuda, "include"),
                     "-c", os.path.join(SRC, f), "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return cmd[-1]

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-ldl", "-lrt", "-lpthread"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
