"""Build libfockx.so in-tree for sm_103a.

Compiles ``csrc/fock_plan.cpp`` with the host compiler, ``csrc/fock_common.cu``
once and ``csrc/fock_kernels_inst.cu`` once per (precision, grid size) listed in
``csrc/fock_sizes.h``, all in parallel, then links them with nvcc.  Objects are
kept under ``_build/`` and rebuilt only when a source or header is newer.

    python -m paper_1305_7313_gb300.build        # or __graft_entry__.build()
"""

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfockx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def grid_sizes():
    text = open(os.path.join(CSRC, "fock_sizes.h")).read()
    m = re.search(r"#define FOCK_GRID_SIZES\(X\)(.*)", text)
    return [int(x) for x in re.findall(r"X\((\d+)\)", m.group(1))]


def _newest_dependency():
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(INCLUDE, "fock.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def _jobs():
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    nv = [nvcc] + ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"] + inc
    jobs = []
    cxx = os.environ.get("CXX", "g++")
    jobs.append(("fock_plan.o", [cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                                 "-I" + os.path.join(cuda, "include")] + inc +
                 ["-c", os.path.join(CSRC, "fock_plan.cpp")]))
    jobs.append(("fock_kpoints.o", [cxx, "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
                                    "-I" + os.path.join(cuda, "include")] + inc +
                 ["-c", os.path.join(CSRC, "fock_kpoints.cpp")]))
    jobs.append(("fock_common.o", nv + ["-c", os.path.join(CSRC, "fock_common.cu")]))
    jobs.append(("fock_static.o", nv + ["-c", os.path.join(CSRC, "fock_static.cu")]))
    jobs.append(("fock_sternheimer.o", nv + ["-c", os.path.join(CSRC, "fock_sternheimer.cu")]))
    for tag, t in (("f64", "double"), ("f32", "float")):
        jobs.append(("fock_persist_%s.o" % tag,
                     nv + ["-DFOCK_T=" + t, "-DFOCK_OPS_NAME=kPersist_%s" % tag,
                           "-c", os.path.join(CSRC, "fock_persist_inst.cu")]))
    for n in grid_sizes():
        for tag, t in (("f64", "double"), ("f32", "float")):
            jobs.append(("fock_%s_%d.o" % (tag, n),
                         nv + ["-DFOCK_T=" + t, "-DFOCK_N=%d" % n, "-DFOCK_OPS_NAME=kOps_%s_%d" % (tag, n),
                               "-DFOCK_KOPS_NAME=kKOps_%s_%d" % (tag, n),
                               "-c", os.path.join(CSRC, "fock_kernels_inst.cu")]))
        # double-float form: Gamma-point kernels only
        jobs.append(("fock_df_%d.o" % n,
                     nv + ["-DFOCK_T=fockx::df64", "-DFOCK_N=%d" % n, "-DFOCK_OPS_NAME=kOps_df_%d" % n,
                           "-c", os.path.join(CSRC, "fock_kernels_inst.cu")]))
    return nvcc, jobs


def build(verbose=False, force=False):
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc, jobs = _jobs()
    newest = _newest_dependency()
    todo = []
    for obj, cmd in jobs:
        out = os.path.join(BUILD, obj)
        if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
            todo.append((out, cmd + ["-o", out]))

    def run(item):
        out, cmd = item
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        return out

    if todo:
        workers = max(1, min(len(todo), os.cpu_count() or 4))
        with cf.ThreadPoolExecutor(workers) as ex:
            for out in ex.map(run, todo):
                if verbose:
                    print("built", os.path.basename(out))
    objs = [os.path.join(BUILD, o) for o, _ in jobs]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
