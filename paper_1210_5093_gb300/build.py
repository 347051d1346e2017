"""Builds libdfamatch.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel; the result is linked with the
static CUDA runtime so the library has no run-time dependency beyond the
driver.  Usage: ``python -m paper_1210_5093_gb300.build`` or ``build()``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libdfamatch.so")
BUILD_DIR = os.path.join(HERE, "_build")
# the debug build: the same sources with DFA_DEBUG_BOUNDS (device-side index checks)
OUT_DEBUG = os.path.join(HERE, "libdfamatch_debug.so")
BUILD_DIR_DEBUG = os.path.join(HERE, "_build_debug")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["dfa_kernels.cu", "dfa_api.cu", "dfa_server.cu", "dfa_noalloc.cu", "dfa_probe.cu",
           "dfa_group.cu",
           "dfa_compile.cpp"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "dfamatch.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _compile(out: str, build_dir: str, extra: list, verbose: bool):
    """Starts the compiles of one library; returns (procs, objs)."""
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I" + CSRC] + extra
    procs, objs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(build_dir, src.rsplit(".", 1)[0] + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, ARCH] + common + ["-c", path, "-o", obj]
        else:
            cmd = [nvcc, "-x", "c++"] + common + ["-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    return procs, objs


def _link(out: str, procs: list, objs: list):
    for cmd, p in procs:
        o, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s" % (" ".join(cmd), o.decode(errors="replace")))
    tmp = out + ".tmp%d" % os.getpid()
    cmd = [_nvcc(), ARCH, "-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stdout.decode(errors="replace")))
    os.replace(tmp, out)


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> str:
    """Builds libdfamatch.so and (debug=True) libdfamatch_debug.so, compiling
    all translation units of both in parallel; returns the release library's path."""
    jobs = []
    if force or _stale(OUT):
        jobs.append((OUT,) + _compile(OUT, BUILD_DIR, [], verbose))
    if debug and (force or _stale(OUT_DEBUG)):
        jobs.append((OUT_DEBUG,) + _compile(OUT_DEBUG, BUILD_DIR_DEBUG, ["-DDFA_DEBUG_BOUNDS"],
                                            verbose))
    for out, procs, objs in jobs:
        _link(out, procs, objs)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
