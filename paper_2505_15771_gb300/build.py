"""Builds libhho.so in-tree with nvcc for sm_103a (GB300).

Host sources are compiled without floating-point contraction so that the
mesh conventions (centroids, diameters, class keys) give the same bits on
x86 and Arm hosts.  Translation units are compiled in parallel.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libhho.so")
PROBE_LIB = os.path.join(HERE, "libhho_probe.so")
SOURCES = ["mesh.cpp", "operators.cpp", "stage.cu", "adjoint.cu", "sdirk.cu", "probe.cu"]

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def _compile(src, verbose):
    out = os.path.join(OBJ, src + ".o")
    cmd = [NVCC] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose and src.endswith(".cu") else []) + \
        ["-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return out, r.stderr


def build(verbose=False):
    os.makedirs(OBJ, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    objs = [o for o, _ in results if not o.endswith("probe.cu.o")]
    probe = [o for o, _ in results if o.endswith("probe.cu.o")]
    if verbose:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", PROBE_LIB] + probe, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("probe link failed:\n%s\n%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
