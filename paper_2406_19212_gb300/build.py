"""Build libgbvqc.so in-tree: every CUDA/C++ source compiled for sm_103a in parallel.

Usage: python -m paper_2406_19212_gb300.build [--force]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbvqc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api_state.cu", "api_matrices.cu", "api_circuit.cu", "api_grad.cu", "api_tune.cu",
           "api_batch.cu", "api_shard.cu", "planner.cpp", "jit.cpp", "kernels_plain.cu", "kernels_reduce.cu",
           "kernels_fused.cu", "kernels_batch.cu", "noalloc.cu"]
# device headers the specialised tile passes are compiled from at run time (NVRTC), embedded
# into the library as strings
JIT_HEADERS = ["common.cuh", "devmath.cuh", "kernels.h", "fused_tile.cuh"]
JIT_DELIM = "GBVQC_JIT_SRC"
# sources compiled as several objects (GBVQC_PART = 0 .. parts-1), one per kernel instance
PARTS = {"kernels_fused.cu": 9, "kernels_batch.cu": 9}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbvqc")


def _flags():
    return ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
            "--expt-relaxed-constexpr"] + ARCH


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gbvqc.h")]
    return max(os.path.getmtime(p) for p in paths)


def _write_jit_headers() -> str:
    """_build/jit_headers.cpp: the JIT_HEADERS as raw string literals (rewritten only when
    their contents change)."""
    parts = ["// generated by build.py: device headers of the specialised tile passes",
             "namespace gbvqc {", f"extern const int kJitHeaderCount = {len(JIT_HEADERS)};",
             "extern const char *const kJitHeaderNames[] = {" + ", ".join(f'"{h}"' for h in JIT_HEADERS) + "};",
             "extern const char *const kJitHeaderSources[] = {"]
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h)).read()
        if f"){JIT_DELIM}\"" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        parts.append(f'R"{JIT_DELIM}({text}){JIT_DELIM}",')
    parts += ["};", "}  // namespace gbvqc", ""]
    out = os.path.join(BUILD, "jit_headers.cpp")
    body = "\n".join(parts)
    if not os.path.exists(out) or open(out).read() != body:
        with open(out, "w") as f:
            f.write(body)
    return out


def _compile(job, verbose: bool) -> str:
    src, part = job
    stem = os.path.splitext(os.path.basename(src))[0] + (f".p{part}" if part is not None else "")
    out = os.path.join(BUILD, stem + ".o")
    defs = [f"-DGBVQC_PART={part}"] if part is not None else []
    path = src if os.path.isabs(src) else os.path.join(CSRC, src)
    cmd = [nvcc()] + _flags() + defs + ["-c", path, "-o", out]
    if src.endswith(".cpp"):
        cmd = [nvcc(), "-x", "cu"] + _flags() + defs + ["-c", path, "-o", out]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"compiling {src} failed:\n{res.stdout}\n{res.stderr}")
    if verbose and res.stderr:
        sys.stderr.write(res.stderr)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libgbvqc.so (skipped when up to date)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = [(_write_jit_headers(), None)]
    for s in SOURCES:
        if os.path.exists(os.path.join(CSRC, s)):
            jobs += [(s, p) for p in range(PARTS[s])] if s in PARTS else [(s, None)]
    # the longest compiles (the kernel instances) first
    jobs.sort(key=lambda j: j[1] is None)
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(4, os.cpu_count() or 4))) as ex:
        objs = list(ex.map(lambda j: _compile(j, verbose), jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-lpthread", "-ldl"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"linking libgbvqc.so failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
