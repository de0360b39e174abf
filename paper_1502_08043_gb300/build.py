"""In-tree build of the CUDA library libcoulomb.so for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel with
    nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo -Xcompiler -fPIC
and linked into paper_1502_08043_gb300/libcoulomb.so (CUDA runtime linked statically).
The seeded input generator's device twin (coulomb_inputs/gen.cu) is built the same way
into coulomb_inputs/libccgen.so.  Rebuilds only when a source or header is newer than
the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libcoulomb.so")
GEN_SRC = os.path.join(ROOT, "coulomb_inputs", "gen.cu")
GEN_LIB = os.path.join(ROOT, "coulomb_inputs", "libccgen.so")

SOURCES = ["tables.cu", "reconstruct.cu", "exchange.cu", "umma.cu", "tcslab.cu", "batched.cu",
           "simtslab.cu", "tcsmall.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libcoulomb")
    return cand


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE)]
    srcs = sources()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + ARCH + FLAGS + ["-I", INCLUDE, "-c", s, "-o", o])
    gen_job = None
    if force or _stale(GEN_LIB, [GEN_SRC]):
        gen_job = [nvcc] + ARCH + FLAGS + ["-shared", GEN_SRC, "-o", GEN_LIB]
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        outs = list(ex.map(_run, jobs + ([gen_job] if gen_job else [])))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    if force or jobs or _stale(LIB, objs):
        _run([nvcc] + ARCH + ["-shared", "-o", LIB] + objs)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
