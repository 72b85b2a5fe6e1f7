"""Compiles the CUDA library (csrc/*.cu) into _lib/libeb_gb300.so for sm_103a.

Translation units compile in parallel with nvcc, then link with -shared.  The
output stays in the source tree (git-ignored) so that the tests and the
benchmark load the library built here.
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libeb_gb300.so")
SOURCES = ["eb_api.cu", "eb_build.cu", "eb_apply.cu", "eb_solve.cu", "eb_noalloc.cu", "eb_mg.cu", "eb_geom.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


TUNED = os.path.join(HERE, "tuned_gb300.json")  # kernel shapes picked by tune.py on a GB300


def tuned_flags(path: str = TUNED) -> list:
    """-D flags of the tuned kernel shapes: the least-squares record's and the apply record's (empty when
    no tuning record exists)."""
    if not os.path.exists(path):
        return []
    with open(path) as f:
        rec = json.load(f)
    best = {**rec.get("best", {}), **rec.get("apply", {}).get("best", {})}
    return [f"-D{k}={int(v)}" for k, v in sorted(best.items())]


def _stale(lib, deps) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, out_dir: str = OUT_DIR, flags=None) -> str:
    """Compile into out_dir/libeb_gb300.so.  flags: extra nvcc flags (default: EB_NVCC_FLAGS from the
    environment, else the tuned kernel shapes)."""
    lib = os.path.join(out_dir, "libeb_gb300.so")
    os.makedirs(os.path.join(out_dir, "obj"), exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "eb.h")]
    if os.path.exists(TUNED):
        deps.append(TUNED)
    if not force and flags is None and not _stale(lib, deps):
        return lib
    if flags is None:
        env = os.environ.get("EB_NVCC_FLAGS")
        flags = env.split() if env is not None else tuned_flags()
    cc = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, "obj", src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
