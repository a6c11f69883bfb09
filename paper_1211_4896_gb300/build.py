"""Builds libvr.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in its own nvcc process (in parallel), then
they are linked into ``_build/libvr.so`` with the static CUDA runtime.
``python -m paper_1211_4896_gb300.build [--verbose] [--checked]`` prints ptxas
resource usage (registers, spills, shared memory) with ``--verbose``;
``--checked`` builds the bounds-check variant ``_build/libvr_checked.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvr.so")
LIB_CHECKED = os.path.join(BUILD, "libvr_checked.so")
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvr.so")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "vr.h"))
    return hs


def _compile(src: str, verbose: bool, checked: bool = False) -> tuple[str, str]:
    obj_dir = os.path.join(BUILD, "checked") if checked else BUILD
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
    if checked:
        cmd.insert(1, "-DVR_BOUNDS_CHECK")
    if src.endswith(".cu"):
        cmd[1:1] = ["-Xptxas", "-v"] if verbose else []
        cmd += ["--expt-relaxed-constexpr"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libvr.so, or with checked=True the bounds-check variant
    libvr_checked.so (-DVR_BOUNDS_CHECK: every gather and scatter index is
    tested against its buffer in the kernels and a violation is reported by
    vr_check instead of being performed)."""
    lib = LIB_CHECKED if checked else LIB
    os.makedirs(os.path.join(BUILD, "checked") if checked else BUILD, exist_ok=True)
    srcs = sources()
    newest = max(os.path.getmtime(p) for p in srcs + _headers() + [__file__])
    if not force and not verbose and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, checked), srcs))
    if verbose:
        for (_, log), src in zip(results, srcs):
            if log.strip():
                print("==", os.path.basename(src))
                print(log)
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv, checked="--checked" in sys.argv))
