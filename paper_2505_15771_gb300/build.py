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
SOURCES = ["mesh.cpp", "operators.cpp", "stage.cu", "adjoint.cu", "sdirk.cu", "tc.cu", "f2x_check.cu", "probe.cu"]

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


def build_stage_variant(tuning_header: str, out_dir: str) -> str:
    """Builds <out_dir>/libhho.so with stage.cu compiled against the given
    stage_tuning.h text (a candidate of tune.py) and the other translation
    units taken from the in-tree build, which must exist."""
    objs = [os.path.join(OBJ, s + ".o") for s in SOURCES if s not in ("stage.cu", "probe.cu")]
    missing = [o for o in objs if not os.path.exists(o)]
    if missing:
        raise RuntimeError("in-tree objects missing (%s); run build() first" % ", ".join(missing))
    src = os.path.join(out_dir, "csrc")
    os.makedirs(src, exist_ok=True)
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            with open(os.path.join(CSRC, f), "rb") as a, open(os.path.join(src, f), "wb") as b:
                b.write(a.read())
    with open(os.path.join(src, "stage_tuning.h"), "w") as f:
        f.write(tuning_header)
    obj = os.path.join(out_dir, "stage.cu.o")
    flags = [x for x in FLAGS if x != "-I" + CSRC] + ["-I" + src]
    r = subprocess.run([NVCC] + ARCH + flags + ["-c", os.path.join(src, "stage.cu"), "-o", obj],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for the stage variant in %s:\n%s" % (out_dir, r.stderr))
    lib = os.path.join(out_dir, "libhho.so")
    r = subprocess.run([NVCC] + ARCH + ["-shared", "-o", lib, obj] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed for the stage variant in %s:\n%s" % (out_dir, r.stderr))
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
