"""Builds the host harness (test infrastructure): the library's host-side
code -- the C ABI, the worker pool, the solver's orchestration, the tuner,
tracing, guard words and the out-of-core executor, compiled as they are --
linked with plain-loop stand-ins for its launchers (stand_ins.cu) and for the
CUDA runtime (stand_in_runtime.cpp) into _build/harness.so, which the CPU
tests load.  Needs nvcc (it cross-compiles; no GPU is used) and g++."""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2408_05238_b300", "csrc")
INC = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "harness.so")
CUDA_INC = "/usr/local/cuda/include"

PRODUCT = ["api.cu", "serving.cu", "solver.cu", "tuner.cu", "trace.cu", "guard.cu", "ooc_solve.cu",
           "ooc_plan.cu"]


def _newer(target: str, deps: list[str]) -> bool:
    return not os.path.exists(target) or any(os.path.getmtime(d) > os.path.getmtime(target)
                                             for d in deps)


def build() -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(INC, f) for f in os.listdir(INC)]
    objs = []
    nvcc = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1",
            "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC]
    for src in [os.path.join(CSRC, f) for f in PRODUCT] + [os.path.join(HERE, "stand_ins.cu")]:
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        if _newer(obj, [src] + headers):
            subprocess.run(nvcc + ["-c", src, "-o", obj], check=True)
        objs.append(obj)
    rt = os.path.join(HERE, "stand_in_runtime.cpp")
    rto = os.path.join(OUT, "stand_in_runtime.o")
    if _newer(rto, [rt]):
        subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-I", CUDA_INC, "-c", rt, "-o", rto],
                       check=True)
    objs.append(rto)
    if _newer(SO, objs):
        # -Bsymbolic: the harness calls its own stand-ins even when the real library,
        # which exports the same names, is already loaded in the process
        subprocess.run(["g++", "-shared", "-Wl,-Bsymbolic", "-o", SO] + objs, check=True)
    return SO


if __name__ == "__main__":
    print(build())
