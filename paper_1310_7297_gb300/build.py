"""In-tree build of libvcm.so and libvcm_checked.so for sm_103a (nvcc, no cmake).

The kernels compile twice - as they are, and with VCM_CHECKED (bounds checks
that set a request's error word instead of making the access) - in parallel
with the host runtime, and link into ``paper_1310_7297_gb300/_build/``:
libvcm.so (the product) and libvcm_checked.so (the checked build the tests
exercise).  A rebuild happens only when a source or header is newer than a
library.
"""

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvcm.so")
LIB_CHECKED = os.path.join(BUILD, "libvcm_checked.so")
SOURCES = ["vcm_kernels.cu", "vcm_api.cpp"]
HEADERS = [os.path.join(CSRC, "vcm_internal.h"), os.path.join(ROOT, "include", "vcm.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code: no contraction into fused multiply-adds, so that host float
# arithmetic (the field-of-view set-up) rounds every operation once.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-Xcompiler", "-ffp-contract=off"]
# (object, source, extra flags)
UNITS = [("vcm_kernels.cu.o", "vcm_kernels.cu", []),
         ("vcm_kernels_checked.cu.o", "vcm_kernels.cu", ["-DVCM_CHECKED"]),
         ("vcm_api.cpp.o", "vcm_api.cpp", [])]
LIBS = [(LIB, ["vcm_kernels.cu.o", "vcm_api.cpp.o"]), (LIB_CHECKED, ["vcm_kernels_checked.cu.o", "vcm_api.cpp.o"])]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def stale():
    if not all(os.path.exists(lib) for lib, _ in LIBS):
        return True
    t = min(os.path.getmtime(lib) for lib, _ in LIBS)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + HEADERS + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Compile libvcm.so and libvcm_checked.so if needed; returns libvcm.so's path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    procs = []
    for obj, src, extra in UNITS:
        cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), cmd))
    errors = []
    for p, cmd in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    if errors:
        raise RuntimeError("libvcm build failed:\n" + "\n".join(errors))
    for lib, objs in LIBS:
        tmp = lib + ".tmp%d" % os.getpid()
        # NVTX loads its tool library by dlopen
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [os.path.join(BUILD, o) for o in objs] + ["-ldl"]
        subprocess.check_call(cmd)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
