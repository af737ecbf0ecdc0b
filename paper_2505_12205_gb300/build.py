"""In-tree build of the CUDA library ``_build/liblbm.so`` for sm_103a.

The translation units (kernels per lattice and storage format, batched-step
kernels, the C ABI of contexts and of batches, the allocation-free
diagnostics, the kernels of the learned fast-forward) are compiled in parallel
with nvcc and linked into a shared library with a static CUDA
runtime.  A content hash of the sources and flags decides whether a rebuild
is needed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
UNITS = ["lbm_d3q19.cu", "lbm_d3q19_f16.cu", "lbm_d3q19_bf16.cu", "lbm_d2q9.cu", "lbm_batch_d2q9.cu",
         "lbm_batch_d3q19.cu", "lbm_api.cu", "lbm_batch.cu", "lbm_noalloc.cu", "nn_kernels.cu"]
HEADERS = ["lbm_lattice.cuh", "lbm_kernels.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
# The lattice Boltzmann units spell every fused multiply-add out (fmaf): with
# contraction left to the compiler, whether a product and a sum fuse depends
# on register pressure, so the same node update compiled for another tile
# shape or register budget would round differently.  With it off, every
# kernel that runs the node update (single contexts, batches of any tile
# width) computes bit-identical results.
NO_CONTRACT = ["-fmad=false"]


def unit_flags(name: str) -> list:
    return FLAGS + ([] if name.startswith("nn_") else NO_CONTRACT)


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _digest() -> str:
    h = hashlib.sha256()
    for name in UNITS + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    for hdr in ("lbm.h", "lbm_nn.h"):
        with open(os.path.join(ROOT, "include", hdr), "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + NO_CONTRACT).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "liblbm.sha256")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    cc = nvcc()

    def compile_unit(name):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        log = os.path.join(BUILD, name.replace(".cu", ".ptxas.log"))
        cmd = [cc] + unit_flags(name) + ARCH + ["-I", os.path.join(ROOT, "include"), "-c",
                                     os.path.join(CSRC, name), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(log, "w") as f:
            f.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (name, r.stderr[-4000:]))
        return obj

    with ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, "-shared"] + ARCH + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
