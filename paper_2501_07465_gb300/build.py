"""Build libpic.so (the CUDA kernels and the C ABI of include/pic.h) in-tree
for sm_103a with nvcc: one object per translation unit, compiled in
parallel, then linked into a shared library next to this file."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpic.so")
SOURCES = ["pic_api.cu", "pic_group.cu", "k_field.cu", "k_field_tma.cu", "k_field_split.cu", "k_field_stream.cu",
           "k_particle.cu", "k_particle_ext.cu", "k_particle_tsc.cu", "k_particle_lean.cu", "k_boundary.cu",
           "k_sort.cu", "k_fd.cu", "k_diag.cu", "k_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, "pic_internal.cuh"), os.path.join(CSRC, "pic_sim.h"),
               os.path.join(CSRC, "k_particle.cuh"),
               os.path.join(INCLUDE, "pic.h")]
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(src: str) -> str:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            cmd = [cc, *ARCH, *FLAGS, "-Xptxas", "-v", *extra, "-c", s, "-o", o]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
            # the register / stack report of every kernel, kept beside the
            # object (tests/test_build_resources.py reads it)
            with open(os.path.join(BUILD, src.replace(".cu", ".ptxas.txt")), "w") as fh:
                fh.write(r.stderr)
            if verbose and r.stderr:
                sys.stderr.write(r.stderr)
        return o

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
