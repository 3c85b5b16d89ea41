"""Build the CUDA library in-tree for sm_103a (nvcc, no cmake).

Two variants of the same sources:

* ``perf`` (``_build/libfasw.so``): the production build, FMA contraction on;
* ``parity`` (``_build_parity/libfasw_parity.so``): ``-fmad=false``, no FMA contraction, so
  that every multiply and add rounds on its own as in a CPU reference compiled without
  contraction.  Only the contraction differs; the kernels and launch shapes are the same.

Translation units compile in parallel; rebuilds only when a source is newer.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
VARIANTS = {
    "perf": (os.path.join(HERE, "_build"), "libfasw.so", []),
    "parity": (os.path.join(HERE, "_build_parity"), "libfasw_parity.so", ["-fmad=false"]),
}
OUT, _name, _ = VARIANTS["perf"]
LIB = os.path.join(OUT, _name)


def lib_path(variant: str = "perf") -> str:
    out, name, _ = VARIANTS[variant]
    return os.path.join(out, name)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(HERE, "..", "include", "fasw.h"), __file__]


def needs_build(variant: str = "perf") -> bool:
    lib = lib_path(variant)
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _deps())


def _start(variant: str, extra: list[str] | None, verbose: bool):
    out, name, vflags = VARIANTS[variant]
    os.makedirs(out, exist_ok=True)
    jobs = []
    for src in _sources():
        obj = os.path.join(out, os.path.basename(src).replace(".cu", ".o"))
        cmd = [NVCC, *FLAGS, *vflags, *(extra or []), "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        jobs.append((obj, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    return jobs


def _finish(variant: str, jobs, verbose: bool) -> str:
    out, name, _ = VARIANTS[variant]
    failed = []
    for obj, cmd, p in jobs:
        text, _ = p.communicate()
        if verbose and text:
            sys.stdout.write(text.decode())
        if p.returncode != 0:
            failed.append((cmd, text.decode()))
    if failed:
        msg = "\n".join(f"{' '.join(c)}\n{o}" for c, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    lib = os.path.join(out, name)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, "-shared", ARCH, "-o", tmp, *[o for o, _, _ in jobs]])
    os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          variant: str = "perf") -> str:
    """Build one variant (when a source is newer than it, or force); returns its path."""
    if not force and not needs_build(variant):
        return lib_path(variant)
    return _finish(variant, _start(variant, extra, verbose), verbose)


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """Both variants, their translation units compiled side by side."""
    todo = [v for v in VARIANTS if force or needs_build(v)]
    started = [(v, _start(v, None, verbose)) for v in todo]
    for v, jobs in started:
        _finish(v, jobs, verbose)
    return [lib_path(v) for v in VARIANTS]


if __name__ == "__main__":
    if "--ptxas" in sys.argv:
        print(build(force=True, verbose=True, extra=["-Xptxas", "-v"]))
    else:
        print(build_all(force="--force" in sys.argv, verbose=True))
