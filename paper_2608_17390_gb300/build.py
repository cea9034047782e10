"""Build libhf.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into
paper_2608_17390_gb300/libhf.so.  Objects go to paper_2608_17390_gb300/_build/.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhf.so")
SOURCES = ["hf_api.cpp", "hf_trace.cu", "hf_pyramid.cu", "hf_march.cu", "hf_scatter.cu", "hf_voxel.cu",
           "hf_serve.cpp", "hf_sun.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, extra=()):
    """Compile and link; returns the library path.  Raises on failure."""
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(ROOT, "include", "hf.h"), os.path.join(CSRC, "hf_internal.h")]
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT, src + ".o")
        objs.append(obj)
        if _stale(obj, [path] + headers) or extra:
            # written under a temporary name and renamed, so that concurrent
            # builds (one per process) never leave a partial object
            tmp = obj + ".tmp%d" % os.getpid()
            cmd = [nvcc()] + _flags() + list(extra) + ["-c", path, "-o", tmp]
            jobs.append((cmd, tmp, obj))

    def run(job):
        cmd, tmp, final = job if isinstance(job, tuple) else (job, None, None)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
        if tmp:
            os.replace(tmp, final)

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB) or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)
