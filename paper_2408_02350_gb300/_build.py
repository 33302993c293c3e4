"""Build libbgk.so (the CUDA library behind include/bgk.h) in-tree with nvcc for sm_103a."""
from __future__ import annotations

import hashlib
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbgk.so")
LIB_DEBUG = os.path.join(HERE, "libbgk_debug.so")
SOURCES = ["abi.cu", "nbr_stencil.cu", "step.cu", "chain.cu", "adjoint.cu", "manage.cu", "noalloc.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
         "-I", CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _stamp(paths: list[str], extra: list[str] | None) -> str:
    """Content hash of the sources, flags and host architecture the library is built from."""
    h = hashlib.sha256()
    for p in sorted(paths):
        h.update(p.encode())
        with open(p, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(ARCH + FLAGS + (extra or [])).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


# Build variants, each a library of its own (libbgk_<name>.so, built in _build_<name>/):
#   debug   every list index a kernel loads checked against the point range (BGK_E_BOUNDS
#           on a bad one, the access skipped);
#   staged  the 2D FP32 transport takes its neighbour rows through per-warp rings of bulk
#           copies into shared memory (transport_stage.cuh) instead of through L1; the same
#           results bit for bit, kept as the measured alternative to the default kernel.
VARIANTS = {"debug": ["-DBGK_DEBUG_BOUNDS=1"],
            "staged": ["-DBGK_WP_STAGE=1", "-DBGK_STAGE_G=4", "-DBGK_STAGE_D=2"]}


def lib_path(variant: str | None = None) -> str:
    return LIB if not variant else os.path.join(HERE, "libbgk_%s.so" % variant)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, debug: bool = False,
          variant: str | None = None) -> str:
    """Build libbgk.so, or the library of one of VARIANTS (debug=True: the bounds-checked
    "debug" one) in a build folder of its own.  Returns the library's path."""
    if debug:
        variant = "debug"
    if variant:
        return _build_into(os.path.join(HERE, "_build_" + variant), lib_path(variant), force, verbose,
                           (extra or []) + VARIANTS[variant])
    return _build_into(BUILD, LIB, force, verbose, extra)


def _build_into(BUILD: str, LIB: str, force: bool, verbose: bool, extra: list[str] | None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(ROOT, "include", "bgk.h"))
    stamp_path = os.path.join(BUILD, "stamp")
    stamp = _stamp([os.path.join(CSRC, s) for s in SOURCES] + headers, extra)
    old = ""
    if os.path.exists(stamp_path):
        with open(stamp_path) as fh:
            old = fh.read()
    if old != stamp or not os.path.exists(LIB):
        force = True
    nvcc = _nvcc()
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, *(extra or []), "-c", s, "-o", o])
    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    with open(stamp_path, "w") as fh:
        fh.write(stamp)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)
