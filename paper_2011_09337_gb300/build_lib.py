"""Builds ``libvit.so`` (the CUDA library behind include/vit.h) in-tree.

Every ``csrc/*.cu`` file is compiled for sm_103a only, in parallel, then
linked into ``paper_2011_09337_gb300/_build/libvit.so``.  Objects are rebuilt
when a source or header is newer than them.

Development aid: ``VIT_BUILD_SKIP`` (comma-separated file stems, e.g.
``vit_codes_k9,vit_codes_k9_bytes,vit_mixed``) leaves those translation
units out of the library, to shorten rebuilds while iterating on other
kernels.  Codes whose kernels are left out are then served by the generic
decoders.  The default build compiles everything.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvit.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _headers() -> list[str]:
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _members_changed(objs: list[str]) -> bool:
    """True when the library was linked from another set of objects."""
    listing = LIB + ".objs"
    want = "\n".join(os.path.basename(o) for o in objs)
    try:
        with open(listing) as fh:
            return fh.read() != want
    except OSError:
        return True


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    skip = {x.strip() for x in os.environ.get("VIT_BUILD_SKIP", "").split(",") if x.strip()}
    srcs = sorted(p for p in glob.glob(os.path.join(CSRC, "*.cu"))
                  if os.path.basename(p)[:-3] not in skip)
    hdrs = _headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [NVCC, *ARCH, *FLAGS, "-c", s, "-o", o + ".tmp"]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stderr}")
        os.replace(o + ".tmp", o)
        return r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for msg in ex.map(compile_one, jobs):
                if verbose and msg:
                    sys.stderr.write(msg)
    if force or jobs or _stale(LIB, objs) or _members_changed(objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(LIB + ".objs", "w") as fh:
            fh.write("\n".join(os.path.basename(o) for o in objs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
