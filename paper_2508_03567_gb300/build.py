"""Compile the CUDA decoder library (libnbldpc.so) in-tree for sm_103a.

The kernel translation units (min-max: one per field order plus the one serving
every field order; FFT-SPA: one per field order) compile in parallel; the host
units hold the C ABI (decoders; serving scheduler and its CUDA executor).
"""
from __future__ import annotations

import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libnbldpc.so")
OBJ_DIR = os.path.join(HERE, "_build")
CSRC = os.path.join(HERE, "csrc")
KERNEL_UNITS = (0, 2, 4, 8, 16, 32, 64, 128, 256)
FFT_UNITS = (2, 4, 8, 16, 32, 64, 128, 256)
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall"]


def _nvcc() -> str:
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(home, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h")) + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def _units():
    units = [(os.path.join(CSRC, "kernels.cu"), f"kernels_q{q}.o", [f"-DNBLDPC_KQ={q}"]) for q in KERNEL_UNITS]
    units += [(os.path.join(CSRC, "fftspa.cu"), f"fftspa_q{q}.o", [f"-DNBLDPC_FQ={q}"]) for q in FFT_UNITS]
    units.append((os.path.join(CSRC, "nbldpc.cu"), "nbldpc.o", []))
    units.append((os.path.join(CSRC, "fftspa_host.cu"), "fftspa_host.o", []))
    units.append((os.path.join(CSRC, "server.cu"), "server.o", []))
    units.append((os.path.join(CSRC, "probe.cu"), "probe.o", []))
    return units


def build_library(force: bool = False, verbose: bool = False, jobs: int | None = None,
                  extra_flags=(), lib_path: str | None = None) -> str:
    """Build libnbldpc.so (or lib_path, with extra nvcc flags such as -D tuning macros)."""
    lib = lib_path or LIB
    if not (force or extra_flags or lib_path or _stale()):
        return lib
    os.makedirs(OBJ_DIR, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    pid = os.getpid()

    def compile_unit(u):
        src, obj, defs = u
        out = os.path.join(OBJ_DIR, f"{pid}_{abs(hash(tuple(extra_flags)))}_{obj}")
        cmd = [nvcc, *NVCC_FLAGS, *inc, *defs, *extra_flags, "-c", src, "-o", out]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return out

    units = _units()
    outs = [os.path.join(OBJ_DIR, f"{pid}_{abs(hash(tuple(extra_flags)))}_{u[1]}") for u in units]
    tmp = lib + f".{pid}.tmp"
    try:
        with ThreadPoolExecutor(max_workers=jobs or min(len(units), os.cpu_count() or 4)) as ex:
            objs = list(ex.map(compile_unit, units))
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", *objs, "-o", tmp])
        os.replace(tmp, lib)
    finally:
        # the objects of this compilation (and a half-written library) go, whether it succeeded or not
        for o in outs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return lib


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
