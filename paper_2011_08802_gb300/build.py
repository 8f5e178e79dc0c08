"""Build of libpfm.so (N = 6 variants) and libpfm_nv12.so (N = 12): every CUDA
translation unit compiled for sm_103a in parallel with nvcc, once per variant
count, then linked into shared libraries in-tree
(``paper_2011_08802_gb300/_lib/libpfm.so``, ``_lib/nv12/libpfm_nv12.so``)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
SOURCES = ["fe_kernels.cu", "mg_kernels.cu", "krylov_kernels.cu", "diag_kernels.cu", "contact_kernels.cu",
           "batch.cu", "api.cu", "noalloc.cu", "params_build.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fno-gnu-unique: function-local statics of templates and inline functions
# become ordinary weak symbols instead of process-wide unique ones, and the
# version script (csrc/exports.map) keeps everything but the C ABI local, so
# libpfm.so and libpfm_nv12.so share no state when one process loads both
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-fno-gnu-unique"]
EXPORTS = os.path.join(CSRC, "exports.map")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


# Libraries built by default: the variant count N of the model is a
# compile-time constant (PFM_NV); N = 6 is the CuAlNi data of Sec. 5.1 and
# N = 12 a NiTi-type variant set (15 unknowns per node).
VARIANTS = {6: ("libpfm.so", ""), 12: ("libpfm_nv12.so", "nv12")}


def lib_path(n_var: int = 6) -> str:
    name, sub = VARIANTS[n_var]
    return os.path.join(OUT, sub, name)


def build(verbose: bool = False, ptxas_info: bool = False, out_dir: str | None = None,
          defines: tuple = (), n_vars: tuple = (6, 12)) -> str:
    """Compile and link one library per variant count in ``n_vars`` (all
    translation units of all of them compiled in parallel); ``out_dir`` and
    ``defines`` build a variant elsewhere (e.g. a launch-configuration sweep)
    without touching the in-tree libraries. Returns the N = 6 library path
    (or the first one built)."""
    jobs = []
    for nv in n_vars:
        name, sub = VARIANTS[nv]
        out = os.path.join(out_dir or OUT, sub)
        os.makedirs(out, exist_ok=True)
        objs = []
        for src in SOURCES:
            obj = os.path.join(out, src.replace(".cu", ".o"))
            cmd = [nvcc(), *ARCH, *FLAGS, f"-DPFM_NV={nv}", *[f"-D{d}" for d in defines], "-c",
                   os.path.join(CSRC, src), "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            objs.append((src, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        jobs.append((os.path.join(out, name), objs))
    failed = []
    for _, objs in jobs:
        for src, _, p in objs:
            log, _ = p.communicate()
            if verbose or p.returncode != 0 or ptxas_info:
                sys.stdout.write(log.decode(errors="replace"))
            if p.returncode != 0:
                failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed for {failed}")
    for lib, objs in jobs:
        tmp = lib + ".tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", *[o for _, o, _ in objs], "-o", tmp, "-lcudart",
                               "-Xlinker", f"--version-script={EXPORTS}"])
        os.replace(tmp, lib)
    return jobs[0][0]


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
