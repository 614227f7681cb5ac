"""Builds liblabs.so (the C-ABI library in csrc/) for sm_103a with nvcc, in-tree.

The translation units compile in parallel; the result lands in _build/liblabs.so
next to this file.  Linking uses the shared CUDA runtime so that the library and
PyTorch share one runtime instance in a process.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblabs.so")
SOURCES = ["labs_walk8a.cu", "labs_walk8b.cu", "labs_walk16a.cu", "labs_walk16b.cu", "labs_walk16p.cu", "labs_walk16q.cu", "labs_walk32.cu", "labs_walk32l.cu", "labs_walk32b.cu", "labs_walk32p.cu", "labs_long.cu", "labs_kernels.cu", "labs_enum.cu", "labs_net.cu", "labs_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblabs")
    return cand


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, h) for h in ("labs_internal.cuh", "labs_device.cuh", "labs_nvtx.h", "labs_async.cuh", "labs_tc.cuh")]
    files += [os.path.join(ROOT, "include", "labs.h"), __file__]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, out: str | None = None) -> str:
    """Compiles the library (to `out`, default _build/liblabs.so); `extra` nvcc flags."""
    if out is None and up_to_date() and not force:
        return LIB
    target = out or LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    flags = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             "-I", CSRC, *(extra or [])]
    if verbose:
        flags += ["-Xptxas", "-v"]
    procs, objs = [], []
    for s in SOURCES:
        obj = os.path.join(OUT_DIR, s.replace(".cu", ".%d.o" % os.getpid()))
        objs.append(obj)
        procs.append((s, subprocess.Popen([cc, *flags, "-c", os.path.join(CSRC, s), "-o", obj],
                                          stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for s, p in procs:
        out, _ = p.communicate()
        if out and (verbose or p.returncode):
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode:
            failed.append(s)
    if failed:
        raise RuntimeError("nvcc failed on " + ", ".join(failed))
    tmp = target + ".%d.tmp" % os.getpid()
    rpath = "-Xlinker=-rpath,/usr/local/cuda/lib64"
    subprocess.run([cc, *ARCH, "-shared", "-cudart", "shared", rpath, *objs, "-o", tmp], check=True)
    os.replace(tmp, target)
    for o in objs:
        os.remove(o)
    return target


if __name__ == "__main__":
    args = sys.argv[1:]
    out = args[args.index("--out") + 1] if "--out" in args else None
    extra = [a for a in args if a.startswith("-D")]
    print(build(force="--force" in args, verbose="-v" in args, extra=extra, out=out))
