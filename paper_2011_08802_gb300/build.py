"""Build of libpfm.so: every CUDA translation unit compiled for sm_103a in
parallel with nvcc, then linked into a shared library in-tree
(``paper_2011_08802_gb300/_lib/libpfm.so``)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
SOURCES = ["fe_kernels.cu", "mg_kernels.cu", "krylov_kernels.cu", "diag_kernels.cu", "contact_kernels.cu",
           "batch.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(verbose: bool = False, ptxas_info: bool = False, out_dir: str | None = None,
          defines: tuple = ()) -> str:
    """Compile and link; ``out_dir``/``defines`` build a variant elsewhere
    (e.g. a launch-configuration sweep) without touching the in-tree library."""
    out = out_dir or OUT
    os.makedirs(out, exist_ok=True)
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(out, src.replace(".cu", ".o"))
        cmd = [nvcc(), *ARCH, *FLAGS, *[f"-D{d}" for d in defines], "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        log, _ = p.communicate()
        if verbose or p.returncode != 0 or ptxas_info:
            sys.stdout.write(log.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    lib = os.path.join(out, "libpfm.so")
    tmp = lib + ".tmp"
    subprocess.check_call([nvcc(), *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
