"""Build the CUDA library ``libflashkin.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` file compiles to an object in ``_build/`` in parallel;
the objects link into one shared library with the CUDA runtime linked
statically.  Sources newer than the library trigger a rebuild.  The variant
"bounds" builds ``libflashkin_bounds.so`` with FK_DEBUG_BOUNDS (the step
kernel checks every index first; the library is loaded instead of the
release one when FK_LIBRARY=bounds is set).
"""
from __future__ import annotations

import glob
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libflashkin.so")
LIBS = {"release": LIB, "bounds": os.path.join(HERE, "libflashkin_bounds.so")}
VARIANT_FLAGS = {"release": [], "bounds": ["-DFK_DEBUG_BOUNDS"]}
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
_lock = threading.Lock()


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def stale(variant: str = "release") -> bool:
    lib = LIBS[variant]
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(),
          variant: str = "release") -> str:
    lib = LIBS[variant]
    out = OUT if variant == "release" else os.path.join(OUT, variant)
    with _lock:
        if not force and not stale(variant):
            return lib
        os.makedirs(out, exist_ok=True)
        procs, objs = [], []
        for src in _sources():
            obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
            cmd = [NVCC, *ARCH, *FLAGS, *VARIANT_FLAGS[variant], *extra_flags, "-c", src, "-o",
                   obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        errors = []
        for src, p in procs:
            out, _ = p.communicate()
            if verbose or p.returncode != 0:
                print(out.decode(errors="replace"))
            if p.returncode != 0:
                errors.append(src)
        if errors:
            raise RuntimeError("nvcc failed for: " + ", ".join(errors))
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call([NVCC, *ARCH, "-shared", "-cudart", "static", *objs, "-ldl",
                               "-o", tmp])
        os.replace(tmp, lib)
    return lib



# The sources the streaming step kernel is compiled from (its DRAM traffic
# recorded under profiles/ stays valid while they are unchanged; the public
# header contributes only enum constants to it).
STEP_KERNEL_SOURCES = (os.path.join(CSRC, "fk_stream.cu"), os.path.join(CSRC, "fk_internal.cuh"))


def code_only(text: str) -> str:
    """C/C++/CUDA source with its comments removed and every run of white
    space made one blank: what the compiler sees, not how it is annotated
    or laid out (string and character literals are kept as they are)."""
    out = []
    i, n = 0, len(text)
    while i < n:
        c = text[i]
        if c == "/" and i + 1 < n and text[i + 1] == "/":
            j = text.find("\n", i)
            i = n if j < 0 else j
            out.append(" ")
        elif c == "/" and i + 1 < n and text[i + 1] == "*":
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def source_hash(files=STEP_KERNEL_SOURCES) -> str:
    """Short hash of the code of the given sources (by default those of the
    streaming step kernel), identifying the code a profile was taken on;
    edits to comments or layout leave it unchanged."""
    import hashlib
    h = hashlib.sha256()
    for p in sorted(files):
        h.update(os.path.basename(p).encode())
        with open(p, encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
