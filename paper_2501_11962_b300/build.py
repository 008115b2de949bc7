"""Builds libmop.so (the CUDA engine behind include/mop.h) in-tree for sm_103a."""
from __future__ import annotations

import os
import subprocess
import sys
from pathlib import Path

HERE = Path(__file__).resolve().parent
CSRC = HERE / "csrc"
LIB = HERE / "libmop.so"
# the same library with the range check of the j-side shares compiled in (for the tests only)
CHECK_LIB = HERE / "libmop_jcheck.so"
SOURCES = ["mop_api.cu", "mop_prep.cu", "mop_pair.cu", "mop_pairb.cu", "mop_path.cu", "mop_pme.cu", "mop_fft.cu",
           "mop_noalloc.cu", "mop_diag.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]
# FP32 subnormals never matter for forces, so the hot kernels flush them (shorter rsqrt path)
PER_FILE = {"mop_pair.cu": ["-ftz=true"], "mop_pairb.cu": ["-ftz=true"], "mop_path.cu": ["-ftz=true"],
            "mop_pme.cu": ["-ftz=true"]}


def _stale(lib: Path = LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = [CSRC / s for s in SOURCES] + list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h"))
    deps.append(HERE.parent / "include" / "mop.h")
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile every .cu into one shared library (objects in parallel, then link)."""
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objdir = HERE / "_build"
    objdir.mkdir(exist_ok=True)
    procs, objs = [], []
    for s in SOURCES:
        obj = objdir / (Path(s).stem + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *PER_FILE.get(s, []), "-c", str(CSRC / s), "-o", str(obj)]
        if verbose:
            print(" ".join(cmd))
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(str(obj))
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed on {s}:\n{out.decode(errors='replace')}")
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [nvcc, *ARCH, "-shared", "-o", str(tmp), *objs, "-lcudart"]
    subprocess.run(cmd, check=True)
    tmp.replace(LIB)
    return LIB


def build_check(force: bool = False) -> Path:
    """libmop_jcheck.so: the objects of build() with mop_pairb.cu compiled with MOP_BL_JCHECK=1."""
    build(force)
    if not force and not _stale(CHECK_LIB):
        return CHECK_LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    objdir = HERE / "_build"
    obj = objdir / "mop_pairb_jcheck.o"
    subprocess.run([nvcc, *ARCH, *FLAGS, *PER_FILE["mop_pairb.cu"], "-DMOP_BL_JCHECK=1", "-c",
                    str(CSRC / "mop_pairb.cu"), "-o", str(obj)], check=True)
    objs = [str(objdir / (Path(s).stem + ".o")) for s in SOURCES if s != "mop_pairb.cu"] + [str(obj)]
    tmp = CHECK_LIB.with_suffix(".so.tmp")
    subprocess.run([nvcc, *ARCH, "-shared", "-o", str(tmp), *objs, "-lcudart"], check=True)
    tmp.replace(CHECK_LIB)
    return CHECK_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    print(build_check(force="--force" in sys.argv))
