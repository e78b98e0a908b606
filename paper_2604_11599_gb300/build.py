"""Builds libsv.so in-tree for sm_103a with nvcc (parallel, no cmake).

    python -m paper_2604_11599_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsv.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["kern_pass.cu", "kern_measure.cu", "kern_batch.cu", "kern_adjoint.cu", "sv_api.cu", "planner.cpp",
           "expval_static.cu", "jit.cpp", "kern_branch.cu", "kern_clifford.cu"]
# headers compiled again at run time by the pass specialiser (jit.cpp); embedded as strings
JIT_HEADERS = [("pass_body.cuh", "csrc/pass_body.cuh"), ("adjoint_body.cuh", "csrc/adjoint_body.cuh"),
               ("batch_body.cuh", "csrc/batch_body.cuh"),
               ("dev_common.cuh", "csrc/dev_common.cuh"),
               ("dev_tc.cuh", "csrc/dev_tc.cuh"),
               ("kernels.h", "csrc/kernels.h"), ("sv_plan.h", "csrc/sv_plan.h"),
               ("../../include/sv.h", "../include/sv.h")]
HEADERS = ["sv_plan.h", "kernels.h", "planner.h", "dev_common.cuh", "dev_tc.cuh", "pass_body.cuh", "adjoint_body.cuh", "batch_body.cuh",
           "jit.h",
           "branch.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "sv.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _embed_jit_headers() -> str:
    """Writes _build/jit_headers.inc: the device headers as string literals."""
    out = os.path.join(BUILD, "jit_headers.inc")
    srcs = [os.path.normpath(os.path.join(HERE, rel)) for _, rel in JIT_HEADERS]
    # the header list lives in this file, so it counts as a source too
    if os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(p) for p in srcs + [__file__]):
        return out
    parts = ["// generated by build.py from the device headers", "static const char* const kJitHeaderNames[] = {"]
    parts += [f'    "{name}",' for name, _ in JIT_HEADERS]
    parts += ["};", "static const char* const kJitHeaderSources[] = {"]
    for p in srcs:
        text = open(p).read()
        if ")SVJIT" in text:
            raise RuntimeError(f"{p} contains the raw-string delimiter")
        parts.append('R"SVJIT(' + text + ')SVJIT",')
    parts += ["};", f"static const int kJitHeaderCount = {len(JIT_HEADERS)};", ""]
    tmp = out + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write("\n".join(parts))
    os.replace(tmp, out)
    return out


def _compile(src: str, verbose_ptxas: bool) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    extra_deps = [os.path.join(BUILD, "jit_headers.inc")] if src == "jit.cpp" else []
    if not _stale(obj, path) and all(os.path.getmtime(d) <= os.path.getmtime(obj) for d in extra_deps):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
           "-I", BUILD, "-c", path, "-o", obj + ".tmp"]
    if src.endswith(".cu"):
        cmd += ["--expt-relaxed-constexpr"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose_ptxas and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for f in os.listdir(BUILD):
            os.remove(os.path.join(BUILD, f))
    _embed_jit_headers()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cuda = os.path.dirname(os.path.dirname(nvcc()))
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart",
               "-L" + os.path.join(cuda, "lib64"), "-lnvrtc",
               "-Xlinker", "-rpath=" + os.path.join(cuda, "lib64")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
