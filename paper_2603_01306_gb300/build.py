"""Builds the CUDA shared libraries in-tree for sm_103a (nvcc, no cmake).

* ``paper_2603_01306_gb300/_lib/librelax.so`` from ``csrc/*.cu`` (the C ABI of
  ``include/relax.h``);
* ``synth/_lib/libsynth.so`` from ``synth/gen.cu`` (seeded input generator).

Translation units are compiled in parallel; a unit is rebuilt only when a
source or header is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-Xcompiler", "-Wno-unused-function"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, obj: str, incs: list[str], extra: list[str], deps: list[str]) -> str:
    if not _newer(obj, [src] + deps):
        return obj
    cmd = [nvcc(), *ARCH, *COMMON, *[f"-I{i}" for i in incs], *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj


def _link(objs: list[str], out: str, libs: tuple = ()) -> None:
    if not _newer(out, objs):
        return
    cmd = [nvcc(), *ARCH, "-shared", "-o", out, *objs, *libs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out}:\n{r.stderr}")


def build(verbose: bool = False, jobs: int | None = None) -> dict:
    csrc = os.path.join(HERE, "csrc")
    libdir = os.path.join(HERE, "_lib")
    objdir = os.path.join(libdir, "obj")
    os.makedirs(objdir, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(csrc, "*.cu")))
    headers = sorted(glob.glob(os.path.join(csrc, "*.cuh"))) + sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
    incs = [csrc, os.path.join(ROOT, "include")]
    synth_src = os.path.join(ROOT, "synth", "gen.cu")
    synth_dir = os.path.join(ROOT, "synth", "_lib")
    os.makedirs(synth_dir, exist_ok=True)
    synth_obj = os.path.join(synth_dir, "gen.o")
    jobs = jobs or max(2, min(len(srcs) + 1, os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(jobs) as ex:
        futs = {ex.submit(_compile, s, os.path.join(objdir, os.path.basename(s)[:-3] + ".o"), incs, [], headers): s
                for s in srcs}
        fsyn = ex.submit(_compile, synth_src, synth_obj, [], [], [])
        objs = [f.result() for f in futs]
        fsyn.result()
    lib = os.path.join(libdir, "librelax.so")
    _link(sorted(objs), lib)
    slib = os.path.join(synth_dir, "libsynth.so")
    _link([synth_obj], slib)
    if verbose:
        print(lib, slib)
    return {"relax": lib, "synth": slib}


if __name__ == "__main__":
    build(verbose=True)
