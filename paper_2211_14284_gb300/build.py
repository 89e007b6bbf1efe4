"""In-tree build of the CUDA extension librm.so for sm_103a (GB300), and of
librm_host.so, the host-only FP64 setup with inspection entry points used by
the CPU tests.

Host sources are compiled with g++, device sources with nvcc, in parallel;
the objects are linked by nvcc into paper_2211_14284_gb300/librm.so.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librm.so")
HOSTLIB = os.path.join(HERE, "librm_host.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SOURCES = ["host_basis.cpp", "host_setup.cpp", "host_probe.cpp"]
DEVICE_SOURCES = ["kernels.cu", "apply_general.cu", "capi.cu", "batch.cu", "learned.cu", "hodge.cu"]
# apply_general_part.cu, once per (space k, first degree of four): the
# compile-time instantiations of the general apply, compiled in parallel;
# apply_cart_part.cu once per space: the Cartesian apply's instantiations
GENERAL_PARTS = [(k, plo) for k in (0, 1, 2) for plo in (1, 5)]
CART_PARTS = [0, 1, 2]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    cmds = []
    objs = []
    for s in HOST_SOURCES:
        o = os.path.join(OUT, s + ".o")
        objs.append(o)
        cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-Wall",
                     "-Wno-unused-function", "-c", os.path.join(CSRC, s), "-o", o])
    units = [(s, s, []) for s in DEVICE_SOURCES]
    units += [("apply_general_part.cu", f"apply_general_k{k}_p{plo}.cu",
               [f"-DRM_GENERAL_K={k}", f"-DRM_GENERAL_PLO={plo}"]) for k, plo in GENERAL_PARTS]
    units += [("apply_cart_part.cu", f"apply_cart_k{k}.cu", [f"-DRM_CART_K={k}"]) for k in CART_PARTS]
    for s, name, defs in units:
        o = os.path.join(OUT, name + ".o")
        objs.append(o)
        cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp", *defs,
               "-c", os.path.join(CSRC, s), "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=len(cmds)) as ex:
        for out in ex.map(_run, cmds):
            logs.append(out)
    probe = os.path.join(OUT, "host_probe.cpp.o")
    solver_objs = [o for o in objs if o != probe]
    logs.append(_run([nvcc, "-shared", *ARCH, "-o", LIB, *solver_objs, "-Xcompiler", "-fopenmp",
                      "-lgomp"]))
    host_objs = [os.path.join(OUT, s + ".o") for s in HOST_SOURCES]
    logs.append(_run(["g++", "-shared", "-fopenmp", "-o", HOSTLIB, *host_objs]))
    text = "\n".join(l for l in logs if l)
    if verbose:
        print(text)
    return text


if __name__ == "__main__":
    print(build(verbose=False, ptxas_info="-v" in sys.argv))
