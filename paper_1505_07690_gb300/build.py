"""Builds libos3d.so (sm_103a) in-tree with nvcc, one object per source file,
compiled in parallel. The library has a plain C ABI (include/os3d.h)."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libos3d.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                  "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest(path, headers):
    h = hashlib.sha256()
    for p in [path] + headers:
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVFLAGS).encode())
    h.update(os.uname().machine.encode())
    return h.hexdigest()[:16]


def build(verbose: bool = False, jobs: int | None = None) -> str:
    """Compiles every .cu under csrc/ and links libos3d.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    headers.append(os.path.join(ROOT, "include", "os3d.h"))
    objs, todo = [], []
    for src in _sources():
        base = os.path.splitext(os.path.basename(src))[0]
        obj = os.path.join(BUILD, f"{base}.{_digest(src, headers)}.o")
        objs.append(obj)
        if not os.path.exists(obj):
            todo.append((src, obj))

    def compile_one(item):
        src, obj = item
        cmd = [nvcc] + NVFLAGS + ["-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        if verbose:
            print(f"compiled {os.path.basename(src)}", file=sys.stderr)
        return obj

    if todo:
        n = jobs or min(len(todo), os.cpu_count() or 4)
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            list(ex.map(compile_one, todo))
    stamp = hashlib.sha256("".join(objs).encode()).hexdigest()[:16]
    stamp_file = LIB + ".stamp"
    if not (os.path.exists(LIB) and os.path.exists(stamp_file)
            and open(stamp_file).read() == stamp):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
        with open(stamp_file, "w") as fh:
            fh.write(stamp)
    # objects of earlier source states are not needed again
    keep = {os.path.basename(o) for o in objs}
    for name in os.listdir(BUILD):
        if name.endswith(".o") and name not in keep:
            try:
                os.remove(os.path.join(BUILD, name))
            except OSError:
                pass
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
