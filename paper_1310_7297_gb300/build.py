"""In-tree build of libvcm.so for sm_103a (nvcc, no cmake).

The two translation units compile in parallel and link into
``paper_1310_7297_gb300/_build/libvcm.so``.  A rebuild happens only when a
source or header is newer than the library.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvcm.so")
SOURCES = ["vcm_kernels.cu", "vcm_api.cpp"]
HEADERS = [os.path.join(CSRC, "vcm_internal.h"), os.path.join(ROOT, "include", "vcm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code: no contraction into fused multiply-adds, so that host float
# arithmetic (the field-of-view set-up) rounds every operation once.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-Xcompiler", "-ffp-contract=off"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile libvcm.so if needed; returns its path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc()] + ARCH + FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), cmd))
        objs.append(obj)
    errors = []
    for p, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    if errors:
        raise RuntimeError("libvcm build failed:\n" + "\n".join(errors))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
