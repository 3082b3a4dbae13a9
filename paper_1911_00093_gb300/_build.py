"""Build libhmat.so in-tree: host C++ (builder, layout) with g++ and the CUDA
sources with nvcc for sm_103a only, compiled in parallel, linked with nvcc."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libhmat.so")
BUILD = os.path.join(HERE, "_build")

CXX_SOURCES = ["builder.cpp", "layout.cpp", "paper_forms.cpp"]
CU_SOURCES = ["kernels.cu", "kernels_table1.cu", "multi.cu", "mrhs.cu", "gmres.cu", "api.cu", "noalloc.cu",
              "aca_device.cu", "multi_df.cu"]
# per-file flags: the device builder reproduces the host builder's rounding (no FMA contraction)
CU_FLAGS = {"aca_device.cu": ["-fmad=false"]}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout)
    return p.stdout


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, s) for s in CXX_SOURCES + CU_SOURCES]
    hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))] + [os.path.join(INCLUDE, "hmat.h")]
    if not force and os.path.exists(OUT):
        newest = max(os.path.getmtime(f) for f in srcs + hdrs + [__file__])
        if os.path.getmtime(OUT) >= newest:
            return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    for s in CXX_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append(([os.environ.get("CXX", "g++"), "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-ffp-contract=off",
                      "-Wall", "-Wno-unknown-pragmas"] + inc +
                     ["-I/usr/local/cuda/include", "-c", os.path.join(CSRC, s), "-o", o], o))
    for s in CU_SOURCES:
        o = os.path.join(BUILD, s + ".o")
        jobs.append(([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                                      "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr"] +
                     CU_FLAGS.get(s, []) + inc +
                     ["-c", os.path.join(CSRC, s), "-o", o], o))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = OUT + f".tmp{os.getpid()}"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + [j[1] for j in jobs] + ["-Xcompiler", "-fopenmp", "-lgomp"])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
