"""Build the CUDA library in-tree: ``libmsim.so`` next to this file, for sm_103a only.

``python -m paper_2603_29332_b300.build`` (or ``__graft_entry__.build()``) runs nvcc once per
changed source set; the result is loaded by :mod:`paper_2603_29332_b300.msim`.
"""
import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmsim.so")
# the same library with every index through the step kernel's views checked (MSIM_BOUNDS_CHECK):
# test infrastructure, the stand-in for a memory checker
CHECK_LIB = os.path.join(HERE, "libmsim_check.so")
SOURCES = ["msim_api.cu", "step_kernels.cu", "gemm_tc.cu", "mlp.cu", "surrogate.cu", "noalloc.cu", "tune.cu", "policy.cu", "peak.cu"]
HEADERS = ["image.h", "kernels.h", "dfloat.cuh", "gemm_tc.h", "mlp.h", "surrogate.h", "handle.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]


# the files that decide the step kernel's code and memory traffic (model image, launch shape)
STEP_FILES = ["step_kernels.cu", "kernels.h", "image.h", "dfloat.cuh", "msim_api.cu"]


def _digest(files=None):
    """SHA-256 of the given csrc files and the compiler flags; by default of all sources and
    headers plus the public headers (the build stamp)."""
    h = hashlib.sha256()
    for f in (SOURCES + HEADERS if files is None else files):
        h.update(open(os.path.join(CSRC, f), "rb").read())
    if files is None:
        for f in ("msim.h", "msim_model.h"):
            h.update(open(os.path.join(ROOT, "include", f), "rb").read())
    h.update(" ".join(ARCH + FLAGS).encode())
    return h.hexdigest()


def step_digest():
    """Digest of the step kernel's sources (keys the committed DRAM-traffic figure)."""
    return _digest(STEP_FILES)


def build(force=False, verbose=False, lib=LIB, defines=()):
    stamp = lib + ".sha256"
    dig = _digest() + " ".join(defines)
    if not force and os.path.exists(lib) and os.path.exists(stamp) and open(stamp).read().strip() == dig:
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = ["nvcc"] + ARCH + FLAGS + list(defines) + ["-I", os.path.join(ROOT, "include"), "-o", tmp] + \
          [os.path.join(CSRC, s) for s in SOURCES] + ["-lcudart"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(dig + "\n")
    return lib


def build_check(force=False, verbose=False):
    """The bounds-checking library (``libmsim_check.so``): every index through the step kernel's
    views of its workspace and model tables is checked; see ``msim_debug_bounds``."""
    return build(force, verbose, CHECK_LIB, ("-DMSIM_BOUNDS_CHECK",))


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
