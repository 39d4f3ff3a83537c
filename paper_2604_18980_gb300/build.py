"""Build libags.so (CUDA, sm_103a) in-tree.

Each translation unit in ``csrc/`` is compiled by its own nvcc process (in
parallel), then linked with ``nvcc -shared``.  The result goes to
``paper_2604_18980_gb300/_build/libags.so``; the CUDA runtime is linked
statically, so the library needs only the driver at run time.

``build(debug=True)`` makes ``libags_debug.so`` beside it, compiled with
``-DAGS_DEBUG``: every index the kernels read from their inputs (pair
values, tile ranges, emission order entries) is checked before it is used; a
failed check records AGS_ERR_BOUNDS in the status block and skips the access
instead of trapping.  The binding loads it when the environment sets
AGS_DEBUG=1.
"""
from __future__ import annotations

import concurrent.futures
import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libags.so")
DEBUG_LIB = os.path.join(BUILD, "libags_debug.so")
DEBUG_FLAGS = ["-DAGS_DEBUG"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


_reported = set()     # "up to date" is logged once per process and library


def _stamp(lib_path: str) -> str:
    return lib_path + ".src-sha256"


def source_digest(extra_flags=None) -> str:
    """SHA-256 over every source and header, the flags, the architecture and
    the host machine: a library whose stamp matches was built from exactly
    these sources here (a copied or stale binary has no matching stamp)."""
    h = hashlib.sha256()
    for p in sorted(_deps()):
        h.update(os.path.relpath(p, HERE).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS + list(extra_flags or [])).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def up_to_date(extra_flags=None, lib_path: str = LIB) -> bool:
    stamp = _stamp(lib_path)
    if not (os.path.exists(lib_path) and os.path.exists(stamp)):
        return False
    with open(stamp) as f:
        return f.read().strip() == source_digest(extra_flags)


def build(force: bool = False, verbose: bool = False, extra_flags=None, quiet: bool = False,
          debug: bool = False) -> str:
    """Compile and link libags.so (libags_debug.so with debug=True) unless the
    stamped build matches the sources; returns its path and logs which of the
    two happened (stderr)."""
    lib_path = DEBUG_LIB if debug else LIB
    extra_flags = (DEBUG_FLAGS if debug else []) + list(extra_flags or [])
    if not force and up_to_date(extra_flags, lib_path):
        if not quiet and lib_path not in _reported:
            print("libags: up to date (%s)" % lib_path, file=sys.stderr)
            _reported.add(lib_path)
        return lib_path
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + extra_flags
    digest = source_digest(extra_flags)
    suffix = ".debug.o" if debug else ".o"

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + suffix)
        cmd = [cc] + ARCH + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib_path + ".tmp%d" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    stamp = _stamp(lib_path)
    with open(stamp + ".tmp", "w") as f:
        f.write(digest)
    os.replace(stamp + ".tmp", stamp)
    if not quiet:
        print("libags: compiled %d translation units (%s)" % (len(objs), lib_path), file=sys.stderr)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
