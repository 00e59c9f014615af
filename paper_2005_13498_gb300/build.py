"""In-tree build of libhubbard_ed.so for sm_103a.

    python -m paper_2005_13498_gb300.build

compiles the CUDA kernels with nvcc (-gencode arch=compute_103a,code=sm_103a)
and the host C++ with g++, in parallel, and links one shared library into
paper_2005_13498_gb300/_lib/.  No CMake.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libhubbard_ed.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["kernels.cu", "docc_static.cu"]
CPP_SOURCES = ["tables.cpp", "engine.cpp", "api.cpp", "drivers.cpp"]


def cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found (set CUDA_HOME)")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" +
                           r.stdout + r.stderr)
    return r.stdout + r.stderr


def lib_path():
    return os.path.join(OUT_DIR, LIB_NAME)


PROBES_NAME = "libed_probes.so"


def probes_path():
    return os.path.join(OUT_DIR, PROBES_NAME)


def build_probes(force=False):
    """libed_probes.so (include/ed_probes.h): the on-chip ceiling probes that
    the benchmark reports beside the roofline."""
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    src = os.path.join(CSRC, "probes.cu")
    hdr = os.path.join(os.path.dirname(HERE), "include", "ed_probes.h")
    target = probes_path()
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(target):
        if os.path.getmtime(target) >= max(os.path.getmtime(src), os.path.getmtime(hdr)):
            return target
    tmp = target + ".tmp"
    _run([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                          "-shared", src, "-o", tmp, "-lcudart",
                          "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")])
    os.replace(tmp, target)
    return target


def build(verbose=False, force=False):
    cuda = cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = os.path.join(cuda, "include")
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in CU_SOURCES + CPP_SOURCES]
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "ed.h"))
    target = lib_path()
    if not force and os.path.exists(target):
        newest = max(os.path.getmtime(p) for p in srcs + headers + [__file__])
        if os.path.getmtime(target) >= newest:
            build_probes()
            return target
    jobs = []
    objs = []
    for s in CU_SOURCES:
        o = os.path.join(BUILD_DIR, s + ".o")
        objs.append(o)
        jobs.append([nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17",
                                     "-Xcompiler", "-fPIC", "-c",
                                     os.path.join(CSRC, s), "-o", o])
    for s in CPP_SOURCES:
        o = os.path.join(BUILD_DIR, s + ".o")
        objs.append(o)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-Wno-unused-function",
                     "-I", inc, "-c", os.path.join(CSRC, s), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs) + 1)) as ex:
        probes = ex.submit(build_probes, force)
        logs = list(ex.map(_run, jobs))
        probes.result()
    if verbose:
        for cmd, log in zip(jobs, logs):
            print(" ".join(cmd))
            if log.strip():
                print(log)
    tmp = target + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs +
         ["-lcudart", "-Xlinker", "-rpath," + os.path.join(cuda, "lib64")])
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
