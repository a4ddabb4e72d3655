"""Build libdpcs.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel to an object file; the shared
library links against the shared CUDA runtime.  Outputs go to
``paper_2503_12174_gb300/_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "lbvh.cu", "render.cu", "optim.cu", "serve.cu", "denoise.cu", "principled.cu", "wavefront.cu",
           "pose.cu"]
# the measurement library (roof probes), used by the benchmark and its tests
PROBE_SOURCES = ["probe.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def lib_path(variant: str = "") -> str:
    return os.path.join(OUT, f"libdpcs{variant}.so")


def _deps(sources=SOURCES):
    return [os.path.join(CSRC, s) for s in sources] + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def build(force: bool = False, variant: str = "", defines=(), verbose: bool = False, sources=None,
          name: str = "libdpcs") -> str:
    """Compile and link; returns the library path.  ``variant`` names an
    alternative build (e.g. "_counters" with defines=("DPCS_COUNTERS",));
    ``sources`` / ``name`` select another library (the probes)."""
    os.makedirs(OUT, exist_ok=True)
    sources = SOURCES if sources is None else sources
    lib = os.path.join(OUT, f"{name}{variant}.so")
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in _deps(sources)):
            return lib
    cc = nvcc()
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
             "--expt-relaxed-constexpr"] + [f"-D{d}" for d in defines]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, f"{os.path.splitext(src)[0]}{variant}.o")
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj, *flags]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{p.stderr}")
        return obj, p.stderr

    with cf.ThreadPoolExecutor(max_workers=len(sources)) as ex:
        results = list(ex.map(compile_one, sources))
    if verbose:
        for _, err in results:
            print(err)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", *ARCH, "-o", tmp, *[o for o, _ in results], "-cudart", "shared"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stderr}")
    os.replace(tmp, lib)
    return lib


def build_probe(force: bool = False) -> str:
    """The measurement library libdpcs_probe.so (roof probes)."""
    return build(force=force, sources=PROBE_SOURCES, name="libdpcs_probe")


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
