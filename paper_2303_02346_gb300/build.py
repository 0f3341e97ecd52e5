"""Build the CUDA library `lib/libmpmsim.so` in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library with a static CUDA runtime. A stamp of the
sources and flags skips the rebuild when nothing changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
BUILD = os.path.join(ROOT, "_build")
LIBNAME = "libmpmsim.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
UNITS = ["sim_api.cu", "kern_fwd.cu", "kern_adj.cu", "kern_misc.cu", "kern_share.cu", "kern_rigid.cu", "noalloc.cu",
         "sur_api.cu", "sur_conv.cu", "sur_wgrad.cu", "sur_kernels.cu", "gas.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found; the CUDA library cannot be built")


def _stamp() -> str:
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


# The sources each kernel family's device code depends on (launchers
# included); host API files are left out, so changing them does not mark
# kernel profiles stale.
KERNEL_SOURCES = {
    "mpm": ["common.cuh", "constitutive.cuh", "scatter.cuh", "tool.cuh", "kernels.h", "kern_fwd.cu",
            "kern_adj.cu"],
    # the forward step kernels alone (sort, P2G, G2P->P2G, grid update, G2P)
    "mpm_fwd": ["common.cuh", "constitutive.cuh", "scatter.cuh", "tool.cuh", "kernels.h", "kern_fwd.cu"],
    # the adjoint kernels (G2P, grid and P2G adjoints, the fused adjoint)
    "mpm_adj": ["common.cuh", "constitutive.cuh", "scatter.cuh", "tool.cuh", "kernels.h", "kern_adj.cu"],
    "surrogate": ["sur_ptx.cuh", "sur_kernels.h", "sur_conv.cu", "sur_wgrad.cu", "sur_kernels.cu"],
    "share": ["common.cuh", "kernels.h", "share.h", "kern_share.cu"],
    "gas": ["gas.cu"],
    "rigid": ["common.cuh", "constitutive.cuh", "rigid.h", "kern_rigid.cu"],
}


def source_hash(group: str = "mpm") -> str:
    """Hash of one kernel family's device sources (machine independent):
    group "mpm" = the simulator's step and adjoint kernels, "mpm_fwd" / "mpm_adj"
    = the step kernels / the adjoint kernels alone, "surrogate" = the
    surrogate's kernels. Profile summaries record it so that stale counters
    can be recognised."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[group]:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    os.makedirs(BUILD, exist_ok=True)
    stamp = _stamp()
    stamp_file = os.path.join(LIBDIR, "build.stamp")
    out = lib_path()
    if not force and os.path.exists(out) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return out
    cc = nvcc()
    procs = []
    objs = []
    for u in UNITS:
        obj = os.path.join(BUILD, u.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + ARCH + FLAGS + ["-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((u, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for u, p in procs:
        o, _ = p.communicate()
        if p.returncode != 0:
            failed.append((u, o.decode(errors="replace")))
        elif verbose and o:
            print(o.decode(errors="replace"))
    if failed:
        msg = "\n".join(f"--- {u} ---\n{o}" for u, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = out + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, out)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
