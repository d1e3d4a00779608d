"""Build libldpc.so in-tree with nvcc for sm_103a (one -gencode, sources compiled in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libldpc.so")
GENCODE = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libldpc.so")
    return cand


def _flags():
    return ["-O3", "-std=c++17", GENCODE, "-lineinfo", "-Xcompiler", "-fPIC",
            "-Xptxas", "-O3", "--expt-relaxed-constexpr", "-I", BUILD]


# Headers the runtime compiler needs for the per-graph batch kernels (pair_jit.cu,
# t16_jit.cu) and the compiled work-list kernels (list_jit.cu), under the names by which
# they are included.
JIT_FILES = (("pair_kernel.cuh", os.path.join(CSRC, "pair_kernel.cuh")),
             ("ll_kernel.cuh", os.path.join(CSRC, "ll_kernel.cuh")),
             ("t16_kernel.cuh", os.path.join(CSRC, "t16_kernel.cuh")),
             ("f16x2.h", os.path.join(CSRC, "f16x2.h")),
             ("ldpc_params.h", os.path.join(CSRC, "ldpc_params.h")),
             ("tmem.h", os.path.join(CSRC, "tmem.h")))
JIT_HEADER = os.path.join(BUILD, "ldpc_jit_sources.h")


def _write_jit_sources() -> None:
    """Embed the kernel headers as string literals (rewritten only when they change)."""
    out = ["// Generated by build.py: the headers of pair_kernel.cuh for the runtime compiler.",
           "#pragma once", "namespace ldpc {", "namespace jitsrc {",
           "struct File { const char *name; const char *text; };",
           "static const File kFiles[] = {"]
    for name, path in JIT_FILES:
        text = open(path).read()
        if ")LDPCSRC" in text:
            raise RuntimeError(f"{path}: contains the raw-string delimiter")
        out.append(f'    {{"{name}", R"LDPCSRC({text})LDPCSRC"}},')
    out += ["};", "}  // namespace jitsrc", "}  // namespace ldpc", ""]
    body = "\n".join(out)
    if not os.path.exists(JIT_HEADER) or open(JIT_HEADER).read() != body:
        tmp = JIT_HEADER + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            f.write(body)
        os.replace(tmp, JIT_HEADER)


def _stale(obj: str, src: str, headers: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src] + headers)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    _write_jit_sources()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.h")) +
                     glob.glob(os.path.join(CSRC, "*.cuh")) +
                     glob.glob(os.path.join(HERE, "..", "include", "*.h")) + [JIT_HEADER])
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, s, headers):
            jobs.append([nvcc, *_flags(), "-c", s, "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
        for j, f in zip(jobs, futs):
            r = f.result()
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(j)}\n{r.stdout}\n{r.stderr}")
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc, GENCODE, "-shared", "-o", tmp, *objs, "-lcudart", "-lnvrtc"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
