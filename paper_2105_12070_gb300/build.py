"""Builds libchemgpu.so (the C-ABI library of include/chemgpu.h) in-tree for sm_103a.

Seven translation units compiled in parallel with nvcc, linked as one shared library:
  csrc/mech_tables.cpp     -- mechanism reader and table layout (host)
  csrc/chem_kernels.cu     -- rate / Jacobian and mapping kernels, launch shapes, CUDA graphs and
                              the extern "C" entry points
  csrc/integrate_g{1,2,4,8}.cu -- the integrate kernels (Rosenbrock, Seulex) for cell groups of
                              1, 2, 4 and 8 warps (device code in csrc/integrate_device.cuh)
  csrc/adjoint.cu          -- the discrete-adjoint kernels (reverse sweep)
(csrc/cell_device.cuh holds the device code the kernel files share.)
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libchemgpu.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["mech_tables.cpp", "chem_kernels.cu", "adjoint.cu", "integrate_g1.cu", "integrate_g2.cu", "integrate_g4.cu",
           "integrate_g8.cu"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "chemgpu.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, defines=(), out: str | None = None) -> str:
    """Compiles the library (into `out`, default the in-tree _build/libchemgpu.so); `defines` are
    extra -D macros (e.g. CHEM_PHASE_TIMERS for the per-phase cycle counters)."""
    lib = out or LIB
    if not force and out is None and not _stale():
        return LIB
    build_dir = os.path.dirname(lib)
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE] + ARCH
    common += [f"-D{d}" for d in defines]
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(build_dir, src + f".{os.getpid()}.o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd[1:1] = ["-x", "cu"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        procs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    failed = []
    for src, p in zip(SOURCES, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = lib + f".{os.getpid()}.tmp"
    subprocess.run([nvcc, "-shared", "-cudart", "static"] + ARCH + ["-o", tmp] + objs, check=True)
    os.replace(tmp, lib)
    for o in objs:
        os.remove(o)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
