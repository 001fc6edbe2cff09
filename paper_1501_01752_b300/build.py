"""Build the in-tree CUDA library ``libgsm.so`` for sm_103a.

    python -m paper_1501_01752_b300.build [--force]

Every translation unit under ``csrc/`` is compiled by nvcc in parallel into
``_build/`` and linked (static CUDA runtime) next to this file, where the
Python binding loads it.  Rebuilds only when a source or header is newer than
the library, and then recompiles only the translation units whose source or
locally included headers (followed through ``#include "..."``) are newer than
their object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgsm.so")
BUILD = os.path.join(HERE, "_build")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I" + os.path.join(ROOT, "include")] + ARCH


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(ROOT, "include", "gsm.h"), __file__]


def up_to_date():
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    if not all(os.path.getmtime(d) <= t for d in _deps()):
        return False
    # objects compiled from older sources (an edit during a build) or missing
    objs = [_obj(s) for s in _sources()]
    if any(os.path.exists(o) and os.path.getmtime(o) > t for o in objs):
        return False
    return not any(os.path.exists(o) and _obj_stale(s) for s, o in zip(_sources(), objs))


def _local_includes(path, seen):
    """path and every header it reaches through #include "..." (resolved
    next to the including file, then in include/)."""
    if path in seen or not os.path.exists(path):
        return seen
    seen.add(path)
    with open(path, errors="replace") as f:
        for line in f:
            t = line.strip()
            if t.startswith("#include") and '"' in t:
                name = t.split('"')[1]
                for base in (os.path.dirname(path), os.path.join(ROOT, "include")):
                    cand = os.path.normpath(os.path.join(base, name))
                    if os.path.exists(cand):
                        _local_includes(cand, seen)
                        break
    return seen


def _obj(src):
    return os.path.join(BUILD, os.path.basename(src) + ".o")


def _obj_stale(src):
    obj = _obj(src)
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in _local_includes(src, set()) | {__file__})


def _compile(src, extra):
    obj = _obj(src)
    cmd = [NVCC] + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=()):
    if not force and up_to_date():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    todo = [s for s in srcs if force or extra or _obj_stale(s)]
    results = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            results = list(ex.map(lambda s: _compile(s, list(extra)), todo))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err, file=sys.stderr)
    objs = [_obj(s) for s in srcs]
    tmp = OUT + ".tmp"
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force="--force" in sys.argv, verbose=v, extra=("-Xptxas", "-v") if v else ()))
