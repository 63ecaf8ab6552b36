"""Build the in-tree C-ABI library ``_build/libelsr.so`` with nvcc (sm_103a).

The translation units compile in parallel, then link into one shared
library.  The persistent GVNS kernels are compiled once per instantiation
(accumulator width x bit-row words x table placement x block bound = 24
objects from elsr_vns_inst.cu, and 4 of the serving kernel from
elsr_srv_inst.cu), so no single object carries all of them.
Only nvcc and the host compiler are needed; no cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libelsr.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["elsr_vns_dispatch.cu", "elsr_kernels.cu", "elsr_abi.cu", "elsr_static.cu",
           "elsr_probe.cu", "elsr_serve.cu"]
HEADERS = ["elsr_row.cuh", "elsr_internal.h", "elsr_vns.cuh"]
# (object suffix, defines) of each GVNS kernel instantiation
VNS_INST = [(f"i{acc[3:5]}_w{nw}_{'s' if ts else 'g'}{maxt}",
             [f"-DELSR_INST_ACC={acc}", f"-DELSR_INST_NW={nw}", f"-DELSR_INST_TS={ts}",
              f"-DELSR_INST_MAXT={maxt}"])
            for acc in ("int32_t", "int64_t") for nw in (1, 2) for ts in (1, 0)
            for maxt in (256, 512, 1024)]

# (object suffix, defines) of each serving-kernel instantiation
SRV_INST = [(f"i{acc[3:5]}_w{nw}", [f"-DELSR_INST_ACC={acc}", f"-DELSR_INST_NW={nw}"])
            for acc in ("int32_t", "int64_t") for nw in (1, 2)]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", CSRC, "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return path


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (when sources changed) and return the library path."""
    os.makedirs(BUILD, exist_ok=True)
    deps_common = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "elsr.h")]
    objs = []
    jobs = []
    units = [(src, src.replace(".cu", ".o"), []) for src in SOURCES]
    units += [("elsr_vns_inst.cu", f"elsr_vns_{suf}.o", defs) for suf, defs in VNS_INST]
    units += [("elsr_srv_inst.cu", f"elsr_srv_{suf}.o", defs) for suf, defs in SRV_INST]
    for src, obj, defs in units:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, obj)
        objs.append(o)
        if force or ptxas_info or _stale(o, [s] + deps_common):
            cmd = [nvcc()] + NVCC_FLAGS + defs + ["-c", s, "-o", o]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    logs = []
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        logs = list(ex.map(run, jobs))
    if verbose or ptxas_info:
        for l in logs:
            print(l)
    if jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
