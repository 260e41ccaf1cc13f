"""Build the C-ABI shared library ``libpolar_express.so`` in-tree.

The CUDA sources are compiled for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), each translation unit in
parallel; the host coefficient solver is compiled with g++ and
``-ffp-contract=off`` so that its FP64 arithmetic is exactly the written
sequence of IEEE operations on every host. The library links the CUDA runtime
statically and resolves the driver's tensor-map encoder at run time, so it
loads on machines without a GPU driver.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(HERE, "lib", "obj")
LIBNAME = "libpolar_express.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I" + INCLUDE] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-I" + INCLUDE]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    cu = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h") or f.endswith(".cuh"))
    hdr.append(os.path.join(INCLUDE, "polar_express.h"))
    return cu, cpp, hdr


def _stamp(cu, cpp, hdr) -> str:
    h = hashlib.sha256()
    for p in cu + cpp + hdr:
        with open(p, "rb") as f:
            h.update(p.encode() + b"\0" + f.read())
    h.update(" ".join(NVCC_FLAGS + CXX_FLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()


def library_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile (if stale) and return the path of the shared library."""
    cu, cpp, hdr = _sources()
    os.makedirs(OBJDIR, exist_ok=True)
    stamp = _stamp(cu, cpp, hdr)
    stamp_file = os.path.join(LIBDIR, ".stamp")
    out = library_path()
    if not force and os.path.exists(out) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read().strip() == stamp:
                return out
    nvcc = _nvcc()
    jobs = []
    objs: List[str] = []
    for src in cu:
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        objs.append(obj)
        cmd = [nvcc, "-c", src, "-o", obj] + NVCC_FLAGS
        jobs.append((cmd, src))
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    for src in cpp:
        obj = os.path.join(OBJDIR, os.path.basename(src) + ".o")
        objs.append(obj)
        jobs.append(([cxx, "-c", src, "-o", obj] + CXX_FLAGS + ["-I" + "/usr/local/cuda/include"], src))
    procs = []
    for cmd, src in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT), src))
    errors = []
    for p, src in procs:
        o, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"--- {src}\n{o.decode(errors='replace')}")
        elif verbose and o:
            print(o.decode(errors="replace"), file=sys.stderr)
    if errors:
        raise RuntimeError("build failed:\n" + "\n".join(errors))
    tmp = out + ".tmp"
    link = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-lpthread", "-ldl", "-lrt"]
    if verbose:
        print(" ".join(link), file=sys.stderr)
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, out)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
