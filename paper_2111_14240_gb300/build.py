"""Build libpmace.so in-tree for sm_103a (GB300) with nvcc.

Every translation unit under csrc/ is compiled in parallel to an object file
in _build/, then linked into paper_2111_14240_gb300/libpmace.so.  Objects are
rebuilt when a source or header is newer.  `python -m
paper_2111_14240_gb300.build` runs it from the command line (`--debug`: the
bounds-checking build, compiled with -DPMACE_DEBUG into libpmace_debug.so).
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libpmace.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", INCLUDE]
# Extra nvcc flags (for example -DPMACE_DEBUG for the bounds-checking build)
# from the environment when build() is not given any; objects built with
# other flags go to their own build folder.
ENV_EXTRA = os.environ.get("PMACE_NVCC_FLAGS", "").split()
DEBUG_FLAGS = ["-DPMACE_DEBUG"]
DEBUG_LIB = os.path.join(PKG, "libpmace_debug.so")


def _build_dir(extra) -> str:
    if not extra:
        return BUILD
    import hashlib
    return BUILD + "_" + hashlib.sha256(" ".join(extra).encode()).hexdigest()[:8]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the PMACE CUDA library cannot be built")


def _newest_dep() -> float:
    deps = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps += glob.glob(os.path.join(INCLUDE, "*.h"))
    return max((os.path.getmtime(p) for p in deps), default=0.0)


def build(verbose: bool = False, force: bool = False, extra=None, lib: str | None = None) -> str:
    """Compile and link the library; `extra`: additional nvcc flags (default
    PMACE_NVCC_FLAGS), `lib`: output path (default libpmace.so)."""
    extra = ENV_EXTRA if extra is None else list(extra)
    lib = lib or LIB
    build_dir = _build_dir(extra)
    nvcc = _nvcc()
    os.makedirs(build_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdr_time = _newest_dep()
    procs = []
    objs = []
    for src in sources:
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), hdr_time)):
            continue
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), flush=True)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    stamp = os.path.join(build_dir, "flags." + os.path.basename(lib))   # flags the library was linked with
    if (force or not os.path.exists(lib) or procs or not os.path.exists(stamp)
            or open(stamp).read() != " ".join(extra)
            or any(os.path.getmtime(o) > os.path.getmtime(lib) for o in objs)):
        tmp = lib + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, lib)
        # the library now matches this flag set only
        for f in glob.glob(os.path.join(PKG, "_build*", "flags." + os.path.basename(lib))):
            if f != stamp:
                os.remove(f)
        with open(stamp, "w") as f:
            f.write(" ".join(extra))
    return lib


def build_debug(verbose: bool = False) -> str:
    """The bounds-checking build (PMACE_DEBUG) as libpmace_debug.so."""
    return build(verbose=verbose, extra=DEBUG_FLAGS, lib=DEBUG_LIB)


if __name__ == "__main__":
    if "--debug" in sys.argv:
        print(build_debug(verbose="-v" in sys.argv))
    else:
        print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
