"""Builds libbpida.so (the C ABI + sm_103a kernels) in-tree with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libbpida.so")
SOURCES = [os.path.join(HERE, "csrc", n) for n in ("bpida.cu", "bpida_noalloc.cu", "bpida_server.cu",
                                                   "bpida_thread.cu", "bpida_pdb.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", n) for n in ("bpida_device.cuh", "bpida_thread.h", "bpida_pdb.h")] + [
    os.path.join(ROOT, "include", "bpida.h")]

NVCC_FLAGS = [
    "-O3", "-std=c++17",
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-lineinfo",
    "-Xcompiler", "-fPIC",
    "-shared",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the translation units in parallel, then links the library."""
    from concurrent.futures import ThreadPoolExecutor

    if not force and not stale():
        return LIB
    tag = "%d" % os.getpid()
    objs = [os.path.join(HERE, "csrc", os.path.basename(src) + "." + tag + ".o") for src in SOURCES]
    compile_flags = [f for f in NVCC_FLAGS if f != "-shared"]

    def compile_one(src_obj):
        src, obj = src_obj
        cmd = [nvcc(), *compile_flags, "-I" + os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)

    tmp = LIB + ".tmp." + tag
    try:
        with ThreadPoolExecutor(len(SOURCES)) as ex:
            list(ex.map(compile_one, zip(SOURCES, objs)))
        subprocess.check_call([nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-Xcompiler", "-fPIC", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    finally:
        for f in objs + [tmp]:
            if os.path.exists(f):
                os.remove(f)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
