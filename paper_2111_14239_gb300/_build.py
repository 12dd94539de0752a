"""Build librklt.so (the C-ABI library) in-tree with nvcc for sm_103a.

Translation units compile in parallel; nothing is installed outside the package
directory.  Used by the package on first import and by the repository's build
entry point.
"""
from __future__ import annotations

import os
import re
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "librklt.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = [
    "rklt_fused_n8.cu", "rklt_fused_n32.cu", "rklt_fused_n16.cu", "rklt_fused_n4.cu", "rklt_reg_n8.cu",
    "rklt_reg_n8b.cu", "rklt_reg_n4.cu", "rklt_fmssim_n8.cu", "rklt_fmssim_n4.cu",
    "rklt_batch.cu", "rklt_sweep.cu", "rklt_split.cu", "rklt_noalloc.cu", "rklt_quant.cu", "rklt_mssim.cu",
    "rklt_plan.cpp", "rklt_serve.cpp",
    "rklt_host.cpp", "rklt_capi.cpp",
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rklt.h")]
    return max(os.path.getmtime(p) for p in paths)


_INCLUDE_RE = re.compile(r'^\s*#\s*include\s+"([^"]+)"', re.M)


def _tu_deps(src: str) -> set:
    """The source file and every quoted include it reaches (paths resolved next to the includer)."""
    seen, todo = set(), [os.path.join(CSRC, src)]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in seen or not os.path.exists(f):
            continue
        seen.add(f)
        with open(f, encoding="utf-8") as fh:
            for inc in _INCLUDE_RE.findall(fh.read()):
                todo.append(os.path.join(os.path.dirname(f), inc))
    return seen


def _obj_current(src: str, obj: str) -> bool:
    return os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in _tu_deps(src))


def up_to_date() -> bool:
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime()


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE] + ARCH

    def compile_one(src: str):
        obj = os.path.join(OUT_DIR, src + ".o")
        if not force and not ptxas_info and _obj_current(src, obj):
            return src, obj, subprocess.CompletedProcess([], 0, "", "")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info and src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, p

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    failed = [(s, p) for s, _, p in results if p.returncode != 0]
    for s, _, p in results:
        if verbose or p.returncode != 0:
            sys.stderr.write(f"--- {s}\n{p.stdout}{p.stderr}")
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(s for s, _ in failed))
    tmp = LIB + ".tmp"
    link = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + [o for _, o, _ in results]
    p = subprocess.run(link, capture_output=True, text=True)
    if p.returncode != 0:
        sys.stderr.write(p.stdout + p.stderr)
        raise RuntimeError("link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
