"""Build the streaming-load library in-tree.

``libstreamload.so`` (the C ABI of ``include/streamload.h``) is compiled from
``csrc/*.cu`` for sm_103a only, one nvcc process per translation unit in
parallel, then linked against the CUDA runtime.  ``libslworkloads.so`` (the
host input generator) is plain C.

    python -m paper_2608_15764_gb300.build [--force] [--verbose]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstreamload.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
              f"-I{os.path.join(ROOT, 'include')}"]
CU_SOURCES = ["api.cu", "k_util.cu", "k_ldg_u32.cu", "k_ldg_f32.cu", "k_ldg_bf16.cu", "k_ldg_fp8.cu",
              "k_cpasync.cu", "k_cpasync_g.cu", "k_cpasync_dyn.cu", "k_tma.cu", "noalloc.cu", "k_batch_ldg.cu", "k_batch_misc.cu", "batch_api.cu",
              "k_ldg_dyn.cu", "k_ldsts.cu", "k_chase.cu", "k_ldg4.cu", "k_two.cu", "k_ldg32.cu", "k_ldg_fixed.cu", "k_cov.cu"]
HEADERS = ["sl_internal.h", "sl_device.cuh", "sl_mbar.cuh", "k_ldg.cuh", "k_batch.cuh", "k_cpasync.cuh",
           os.path.join("..", "..", "include", "streamload.h")]


def _code_only(text: str) -> str:
    """C/C++ source without its comments and with whitespace runs collapsed
    (the kernel sources hold no comment markers inside string literals)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash() -> str:
    """Hash of the kernel code (csrc/k_*, *.cuh, sl_internal.h, comments and
    layout left out): counters taken on another version of the kernels' code
    are not reported against these."""
    import hashlib
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        if name.startswith("k_") or name.endswith(".cuh") or name == "sl_internal.h":
            with open(os.path.join(CSRC, name), encoding="utf-8") as f:
                h.update(name.encode() + b"\0" + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _nvcc() -> str:
    for cand in [shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _cuda_lib_dir(nvcc: str) -> str:
    root = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    for sub in ["lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
                os.path.join("targets", "x86_64-linux", "lib")]:
        d = os.path.join(root, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(root, "lib64")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA translation unit for sm_103a and link the library.
    Returns the library path.  Raises RuntimeError on a compile error."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in HEADERS]
    jobs = []
    for src in CU_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            jobs.append((s, o))

    def compile_one(job):
        s, o = job
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", s, "-o", o + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        log = os.path.join(BUILD, os.path.basename(s) + ".ptxas.log")
        with open(log, "w") as f:
            f.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr[-4000:]}")
        os.replace(o + ".tmp", o)
        return s

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), max(2, os.cpu_count() or 2))) as ex:
            for s in ex.map(compile_one, jobs):
                if verbose:
                    print("compiled", os.path.relpath(s, ROOT))
    objs = [os.path.join(BUILD, src.replace(".cu", ".o")) for src in CU_SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, f"-L{_cuda_lib_dir(nvcc)}", "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
    from . import workloads
    workloads.build(force=force)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    a = ap.parse_args(argv)
    print(build(force=a.force, verbose=a.verbose))


if __name__ == "__main__":
    sys.exit(main())
