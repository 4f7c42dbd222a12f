"""Build the CUDA shared libraries behind include/*.h in-tree for sm_103a.

nvcc cross-compiles without a GPU, so this runs on any machine with CUDA 13.
The libraries land in paper_2303_08123_b300/_lib/ and travel with the source
tree; nothing is installed elsewhere.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

# one shared library per entry translation unit: (sources, extra nvcc flags)
TARGETS = {
    "libsim.so": (["sim_api.cu"], []),
    "libmlp.so": (["mlp_api.cu"], []),
    "libga.so": (["ga_api.cu"], []),
    # debug variant of libsim: every kernel's site indices checked, violations reported in the status word
    "libsim_check.so": (["sim_api.cu"], ["-DSIM_CHECK"]),
}


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])


def build(force: bool = False, verbose: bool = False) -> list:
    """Compile every stale library; the nvcc runs proceed in parallel."""
    os.makedirs(LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _deps())
    out, jobs = [], []
    for lib, (srcs, flags) in TARGETS.items():
        dst = os.path.join(LIBDIR, lib)
        out.append(dst)
        if not force and os.path.exists(dst) and os.path.getmtime(dst) >= newest:
            continue
        tmp = dst + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-cudart", "shared", "-I", os.path.join(ROOT, "include"), *flags, "-o", tmp,
               *[os.path.join(CSRC, s) for s in srcs]]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        jobs.append((subprocess.Popen(cmd), cmd, tmp, dst))
    failed = None
    for proc, cmd, tmp, dst in jobs:
        if proc.wait() != 0:
            failed = failed or subprocess.CalledProcessError(proc.returncode, cmd)
            if os.path.exists(tmp):
                os.remove(tmp)
        else:
            os.replace(tmp, dst)
    if failed:
        raise failed
    return out


if __name__ == "__main__":
    for p in build(force="--force" in sys.argv, verbose="-v" in sys.argv):
        print(p)
