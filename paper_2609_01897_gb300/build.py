"""Build libvista.so in-tree for sm_103a.

The translation units are compiled in parallel (the CUDA sources, with the
stacking kernel's instantiations split by visibility type, and one host C++
file), then linked into paper_2609_01897_gb300/libvista.so with the CUDA
runtime linked statically.  The host planner is compiled with -ffp-contract=off so its FP64
tables are the separately rounded operations the source spells out.
"""
import fcntl
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvista.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["vista_stack_c64.cu", "vista_stack_c128.cu", "vista_stack_f16.cu", "vista_stack_bf16.cu",
              "vista_stack.cu", "vista_kernels.cu", "vista_order.cu", "vista_run.cu", "vista_api.cu", "vista_regrid.cu",
              "vista_noalloc.cu", "vista_autotune.cu", "vista_contsub.cu"]
CXX_SOURCES = ["planner.cpp"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libvista needs the CUDA toolkit to build")


def _sources():
    out = [os.path.join(CSRC, f) for f in CU_SOURCES + CXX_SOURCES]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    out.append(os.path.join(INCLUDE, "vista.h"))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # one builder at a time (several ranks of one job may call this at once);
    # the others find the library up to date once they get the lock
    with open(os.path.join(BUILD, ".lock"), "w") as lk:
        try:
            fcntl.flock(lk, fcntl.LOCK_EX)
        except OSError:   # a filesystem without locks: build unserialised
            pass
        try:
            if not force and up_to_date():
                return LIB
            return _build(verbose)
        finally:
            try:
                fcntl.flock(lk, fcntl.LOCK_UN)
            except OSError:
                pass


def _build(verbose: bool) -> str:
    nvcc = _nvcc()
    inc = ["-I" + INCLUDE, "-I" + CSRC]
    jobs, objs = [], []
    for f in CU_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-Xptxas", "-v" if verbose else "-O3", *inc, "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    for f in CXX_SOURCES:
        obj = os.path.join(BUILD, f + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", *inc,
               "-I" + os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include"),
               "-c", os.path.join(CSRC, f), "-o", obj]
        jobs.append(subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True))
        objs.append(obj)
    failed = []
    for j in jobs:
        out, _ = j.communicate()
        if verbose and out:
            sys.stdout.write(out)
        if j.returncode != 0:
            failed.append(" ".join(j.args) + "\n" + out)
    if failed:
        raise RuntimeError("libvista build failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libvista link failed:\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
