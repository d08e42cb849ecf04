"""Build the CUDA library in-tree: ``_build/libadjtx.so`` for sm_103a.

Regenerates the fast-core header, compiles every ``csrc/*.cu`` translation unit with
nvcc in parallel and links them into one shared library.  Up-to-date objects are kept.
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libadjtx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the adjtx CUDA library cannot be built")


def _flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH


def _newest_dep():
    newest = 0.0
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                newest = max(newest, os.path.getmtime(os.path.join(d, f)))
    return newest


def build(verbose: bool = False, force: bool = False) -> str:
    """Build (if needed) and return the path of libadjtx.so."""
    subprocess.run([sys.executable, os.path.join(CSRC, "gen_cores.py")], check=True)
    os.makedirs(BUILD, exist_ok=True)
    nvcc = nvcc_path()
    srcs = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    dep = _newest_dep()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, s[:-3] + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < dep:
            cmd = [nvcc] + _flags() + ["-Xptxas", "-v", "-c", os.path.join(CSRC, s), "-o", o]
            jobs.append((s, cmd, o + ".ptxas.log"))

    def run(job):
        name, cmd, log = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(log, "w") as f:
            f.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {name}:\n{r.stderr[-4000:]}")
        return name

    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for name in ex.map(run, jobs):
            if verbose:
                print("compiled", name)
    if force or jobs or not os.path.exists(LIB):
        cmd = [nvcc, "-shared"] + ARCH + ["-o", LIB] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
