"""Build the CUDA library libse2.so in-tree (paper_2504_05149_gb300/lib/).

Every translation unit is compiled for sm_103a only, in parallel, then linked
with `nvcc -shared`.  A unit is recompiled when it or any header changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIB = os.path.join(LIBDIR, "libse2.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


SIZES = (8, 16, 32, 64, 128, 256, 512)
FAST_SIZES = (32, 64, 128, 256)


def units():
    """(source, object name, extra flags): se2_inst.cu once per (type, N)."""
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        src = os.path.join(CSRC, f)
        if f == "se2_inst.cu":
            for t in ("float", "double"):
                for n in SIZES:
                    out.append((src, f"se2_inst_{t}_{n}.o", [f"-DSE2_T={t}", f"-DSE2_N={n}"]))
        elif f == "se2_fast.cu":
            for n in FAST_SIZES:
                out.append((src, f"se2_fast_{n}.o", [f"-DSE2_FN={n}"]))
        else:
            out.append((src, f + ".o", []))
    return out


def _headers_mtime() -> float:
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    ts += [os.path.getmtime(os.path.join(INCLUDE, f)) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max(ts) if ts else 0.0


def _compile(unit, extra) -> str:
    src, name, defs = unit
    obj = os.path.join(OBJDIR, name)
    cmd = [_nvcc(), *ARCH, *FLAGS, *defs, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(OBJDIR, exist_ok=True)
    hdr = _headers_mtime()
    todo, objs = [], []
    for u in units():
        obj = os.path.join(OBJDIR, u[1])
        objs.append(obj)
        if force or not os.path.exists(obj) or os.path.getmtime(obj) < max(os.path.getmtime(u[0]), hdr):
            todo.append(u)
    # drop objects of units that no longer exist
    keep = {os.path.basename(o) for o in objs}
    for f in os.listdir(OBJDIR):
        if f.endswith(".o") and f not in keep:
            os.remove(os.path.join(OBJDIR, f))
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for obj in ex.map(lambda u: _compile(u, list(extra)), todo):
                if verbose:
                    print("built", obj, file=sys.stderr)
    if todo or not os.path.exists(LIB):
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart", "-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
