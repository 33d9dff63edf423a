"""Builds libvdbc.so (the C ABI of include/vdbc.h) in-tree with nvcc for sm_103a.

Translation units are compiled in parallel and linked with `nvcc -shared`.
The output lands in paper_2504_04564_gb300/_build/ (git-ignored).
``build(checked=True)`` builds the same sources with VDBC_CHECKED=1 and
VDBC_STATS into _build/checked/libvdbc_checked.so: every tree lookup
bounds-checks its node, leaf and tile indices and reports a violation through
the device error word, and the tracker counts its events (loop iterations,
DDA cells, coarse blocks, free flights, ray starts, paths fetched).
``build(sanitize=True)`` builds _build/asan/libvdbc_asan.so, whose host code
is instrumented by AddressSanitizer and UndefinedBehaviorSanitizer (load it
into a process that starts with libasan preloaded).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libvdbc.so")
BUILD_CHECKED = os.path.join(BUILD, "checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libvdbc_checked.so")
BUILD_ASAN = os.path.join(BUILD, "asan")
LIB_ASAN = os.path.join(BUILD_ASAN, "libvdbc_asan.so")
# (nvcc splits -Xcompiler values at commas: one sanitizer per flag)
SANITIZE_LINK = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"]
SANITIZE_FLAGS = ["-g", "-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=all"] + SANITIZE_LINK
INCLUDE = os.path.join(ROOT, "include")

SOURCES = ["encode.cu", "render.cu", "util.cu", "learn.cu"]
# render.cu fuses multiply-adds only where the source says so (__fmaf_rn), so
# every sampler instantiation of the tracker computes the same bits (free:
# the tracker with contraction on measured 16.13 against 16.15 ms)
PER_FILE_FLAGS = {"render.cu": ["--fmad=false"]}
HEADERS = ["vdbc_device.cuh", "vdbc_host.h", "learn.cuh"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-I" + INCLUDE, "-I" + CSRC]


def _deps():
    return ([os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS] +
            [os.path.join(INCLUDE, "vdbc.h")])


def _variant(checked: bool, sanitize: bool):
    """(library, object folder, extra compile flags, extra link flags)."""
    if checked:
        return LIB_CHECKED, BUILD_CHECKED, ["-DVDBC_CHECKED=1", "-DVDBC_STATS"], []
    if sanitize:
        return LIB_ASAN, BUILD_ASAN, SANITIZE_FLAGS, SANITIZE_LINK
    return LIB, BUILD, [], []


def stale(checked: bool = False, sanitize: bool = False) -> bool:
    lib = _variant(checked, sanitize)[0]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.exists(d) and os.path.getmtime(d) > t for d in _deps())


def build(verbose: bool = False, force: bool = False, extra_flags=None, checked: bool = False,
          sanitize: bool = False) -> str:
    """Compile every translation unit in parallel, then link the shared library
    (the bounds-checked variant with ``checked=True``, the host-sanitized one
    with ``sanitize=True``)."""
    lib, out, vflags, lflags = _variant(checked, sanitize)
    if not force and not stale(checked, sanitize):
        return lib
    os.makedirs(out, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or []) + vflags
    if verbose:
        flags = flags + ["-Xptxas", "-v"]
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(out, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = ["nvcc"] + flags + PER_FILE_FLAGS.get(src, []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode()))
        if verbose and out:
            sys.stdout.write(out.decode())
    tmp = lib + ".tmp"
    cmd = ["nvcc"] + ARCH + lflags + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stdout.decode()))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, checked="--checked" in sys.argv,
                sanitize="--sanitize" in sys.argv))
