"""Build libopstile.so for sm_103a with nvcc (in-tree, no cmake).

Every translation unit is compiled in parallel with
`-gencode arch=compute_103a,code=sm_103a -lineinfo -fmad=false`; the shared
library links the CUDA runtime dynamically so that it shares the process's
CUDA runtime (and primary context) with PyTorch.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from typing import List

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.environ.get("OPSTILE_BUILD_DIR") or os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libopstile.so")

SOURCES = ["runtime.cpp", "plan.cpp", "chain_kernels.cu", "cg.cu", "serve.cpp", "noalloc.cu", "jit.cpp", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build opstile")


def _cuda_lib_dir(nvcc: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "lib64")


def sources() -> List[str]:
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "opstile.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def _embed_device_common(gen_dir: str) -> None:
    """device_common.cuh as a C++ raw string literal, for the run-time compiler."""
    os.makedirs(gen_dir, exist_ok=True)
    text = open(os.path.join(CSRC, "device_common.cuh")).read()
    assert ')DCOMMON"' not in text
    out = os.path.join(gen_dir, "device_common.inc")
    body = "// generated by _build.py from csrc/device_common.cuh\nR\"DCOMMON(" + text + ")DCOMMON\"\n"
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    obj_dir = os.path.join(BUILD, "obj")
    gen_dir = os.path.join(BUILD, "gen")
    os.makedirs(obj_dir, exist_ok=True)
    _embed_device_common(gen_dir)
    common = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "--extended-lambda", "-Xcompiler",
              "-fPIC,-O2,-ffp-contract=off",
              "-I", INCLUDE, "-I", CSRC, "-I", gen_dir] + ARCH
    # optional tuning macros, e.g. OPSTILE_NVCC_DEFS="OPS_PTS=2 OPS_MIN_CTAS=2"
    common += ["-D" + d for d in os.environ.get("OPSTILE_NVCC_DEFS", "").split()]

    def compile_one(src: str) -> str:
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + common
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    libdir = _cuda_lib_dir(nvcc)
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared", "-ldl", "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
