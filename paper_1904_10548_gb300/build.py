"""In-tree build of librapidnet.so for sm_103a with nvcc (no cmake).

Translation units are compiled in parallel into ``_build/`` and linked
into ``librapidnet.so`` next to this file.  The CUDA runtime is linked
statically, so the library needs only the CUDA driver at run time.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "librapidnet.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, extra flags): the kernel units are compiled once per
# component count C and, for the solve and mixed kernels, once per kind of
# W_u (RN_DENSE: 0 diagonal, 1 dense); dispatch.cu chooses the
# instantiation at run time.  The device compiler thus runs on them in
# parallel; the longest compiles (batched, then mixed kernels) are
# submitted first so that the slowest one starts at once.
SOURCES = [("batch_kernels.cu", f"batch_kernels_c{c}.o", [f"-DRN_CVAL={c}"]) for c in (8, 4, 2, 1)]
SOURCES += [(k, f"{os.path.splitext(k)[0]}_c{c}_d{d}.o", [f"-DRN_CVAL={c}", f"-DRN_DENSE={d}"])
            for k in ("mixed_kernels.cu", "solve_kernels.cu") for d in (0, 1)
            for c in (8, 4, 2, 1)]
SOURCES += [(s, os.path.splitext(s)[0] + ".o", []) for s in
            ["pernode.cu", "rapidnet.cu", "dispatch.cu", "scenario_tree.cu", "server.cpp",
             "plan.cpp", "factor_check.cpp", "layout.cpp", "pernode_factor.cpp"]]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _compile(entry, verbose: bool) -> str:
    src, objname, extra = entry
    obj = os.path.join(BUILD, objname)
    path = os.path.join(CSRC, src)
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(INCLUDE, "rapidnet.h"))
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps):
        return obj
    cmd = [_nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", *extra,
           "-I", INCLUDE, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and (r.stdout or r.stderr):
        print(r.stdout, r.stderr)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    workers = max(1, min(len(SOURCES), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
