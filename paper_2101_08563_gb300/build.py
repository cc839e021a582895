"""Builds libfastfca.so (the CUDA library behind include/fastfca.h) in-tree with nvcc.

    python -m paper_2101_08563_gb300.build          # or: from ... import build; build.build()

Translation units compile in parallel, one -gencode (sm_103a), then link into a shared
library next to this file.  A rebuild happens only when a source or header is newer than
the library.  ptxas's per-kernel resource report (registers, spills, stack) is kept in
_build/ptxas_report.json.
"""
from __future__ import annotations

import concurrent.futures as cf
import json
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_NAME = "libfastfca.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)
REPORT_PATH = os.path.join(BUILD_DIR, "ptxas_report.json")

SOURCES = ["fastfca_m4_hi.cu", "fastfca_m4.cu", "fastfca_m3.cu", "fastfca_m2.cu", "api.cu", "fca_ops.cu", "noalloc.cu", "batch.cu",
           "fastmnmf_m2.cu", "fastmnmf_m3.cu", "fastmnmf_m4.cu", "fastmnmf_common.cu",
           "learn.cu", "fastfca_cluster_lo.cu", "fastfca_cluster_hi.cu", "fastfca_sm.cu", "probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", os.path.join(ROOT, "include")]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfastfca.so")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    files.append(os.path.join(ROOT, "include", "fastfca.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB_PATH):
        return False
    t = os.path.getmtime(LIB_PATH)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def parse_ptxas(text: str) -> dict:
    """{mangled kernel name: {"registers", "spill_stores", "spill_loads", "stack"}} from the
    output of ptxas -v."""
    out, cur = {}, None
    for line in text.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            cur = m.group(1)
            out[cur] = {"registers": None, "spill_stores": 0, "spill_loads": 0, "stack": 0}
            continue
        if cur is None:
            continue
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            out[cur]["stack"], out[cur]["spill_stores"], out[cur]["spill_loads"] = (int(g) for g in m.groups())
        m = re.search(r"Used (\d+) registers", line)
        if m:
            out[cur]["registers"] = int(m.group(1))
    return out


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every translation unit for sm_103a and link libfastfca.so; returns its path."""
    if not force and up_to_date():
        return LIB_PATH
    nvcc = nvcc_path()
    os.makedirs(BUILD_DIR, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, "-Xptxas=-v", *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj, parse_ptxas(r.stdout + r.stderr)

    jobs = jobs or min(len(SOURCES), os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    report = {}
    for _, rep in results:
        report.update(rep)
    with open(REPORT_PATH, "w") as f:
        json.dump(report, f, indent=0, sort_keys=True)
    tmp = LIB_PATH + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
