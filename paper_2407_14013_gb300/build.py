"""Build the in-tree CUDA library libwcipm.so for sm_103a with nvcc (no cmake).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  A second library, libwcipm_checked.so, is the
bounds-checked debug build: the translation units that address arrays through
index tables (CHECKED_SOURCES) compiled again with -DSDP_CHECK_BOUNDS and linked
with the other objects (sdp_bounds_report reads its records).  Used by
``__graft_entry__.build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwcipm.so")
LIB_CHECKED = os.path.join(HERE, "libwcipm_checked.so")
CHECKED_SOURCES = ("sparse.cu",)   # gathers and scatters through the sparse operator's index tables
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, extra, tag: str = "") -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + tag + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(LIB_CHECKED)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "wcipm.h"))
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    checked = [s for s in srcs if os.path.basename(s) in CHECKED_SOURCES]
    jobs = [(s, list(extra), "") for s in srcs] + [(s, [*extra, "-DSDP_CHECK_BOUNDS"], "_checked") for s in checked]
    # the longest translation units first, so that the parallel compile ends sooner
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        built = dict(zip([(j[0], j[2]) for j in jobs], ex.map(lambda j: _compile(*j), jobs)))
    objs = [built[(s, "")] for s in srcs]
    objs_checked = [built[(s, "_checked")] if s in checked else built[(s, "")] for s in srcs]
    for lib, o in ((LIB, objs), (LIB_CHECKED, objs_checked)):
        tmp = lib + ".tmp"
        res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *o], capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
        os.replace(tmp, lib)
        if verbose:
            print(f"built {lib}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
