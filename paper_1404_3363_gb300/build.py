"""Build libivv.so (the C-ABI library) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1404_3363_gb300/_build/libivv.so``.  No cmake; one -gencode.
"""
import concurrent.futures as cf
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libivv.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
            "--expt-relaxed-constexpr", "-I", INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I", INCLUDE]

CU_SOURCES = ["ivv_api.cu", "k_surface.cu", "k_pair.cu", "k_integrate_p2.cu", "k_integrate_p3.cu",
              "k_eval.cu", "host_debug.cu", "k_mlp.cu", "k_mlp_tc.cu", "k_rf.cu", "batch.cu", "k_batch.cu",
              "k_integrate_batch.cu", "k_fixed_p2.cu", "k_fixed_p3.cu"]
CXX_SOURCES = ["host_prep.cpp"]


def _deps_hash():
    h = hashlib.sha256()
    for name in sorted(os.listdir(SRC_DIR)):
        if name.endswith((".cu", ".cuh", ".cpp", ".h")):
            with open(os.path.join(SRC_DIR, name), "rb") as f:
                h.update(name.encode() + f.read())
    with open(os.path.join(INCLUDE, "ivv.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + CU_FLAGS + CXX_FLAGS).encode())
    return h.hexdigest()


def _compile(src, extra_flags=()):
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    path = os.path.join(SRC_DIR, src)
    if src.endswith(".cu"):
        cmd = [NVCC] + ARCH + CU_FLAGS + list(extra_flags) + ["-c", path, "-o", obj]
    else:
        cmd = [NVCC, "-x", "c++", "-Xcompiler", "-fPIC", "-O2", "-std=c++17", "-I", INCLUDE, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, ptxas_v=False):
    """Compile (if sources changed) and return the path of libivv.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    stamp = os.path.join(OUT_DIR, "stamp")
    digest = _deps_hash()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    extra = ["-Xptxas", "-v"] if ptxas_v else []
    srcs = CU_SOURCES + CXX_SOURCES
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    if verbose or ptxas_v:
        for obj, log in results:
            if log:
                print(log, file=sys.stderr)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv))
