"""Build libzinc.so (sm_103a) in-tree: paper_2408_07304_gb300/_build/libzinc.so.

Each translation unit compiles in parallel (nvcc for .cu, g++ for the host
tables with -ffp-contract=off), then nvcc links the shared library.  Objects
are rebuilt only when a source or header is newer.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libzinc.so")

CU_SOURCES = ["zn_encrypt.cu", "zn_encrypt_mp.cu", "zn_encrypt_occ.cu", "zn_encrypt_occ3.cu", "zn_encrypt_quarter.cu", "zn_encrypt_pair.cu", "zn_encrypt_ms.cu", "zn_encrypt_int.cu", "zn_zinc_ntt.cu", "zn_bencode.cu", "zn_pack.cu", "zn_batch.cu", "zn_keys.cu", "zn_codec.cu", "zn_probe.cu", "zn_api.cu"]
CPP_SOURCES = ["zn_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzinc.so")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "zinc.h"))
    return hs


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + _headers())


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        objs.append(obj)
        if _stale(obj, src):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--extended-lambda",
                         "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE,
                         "-c", src, "-o", obj] + (["-Xptxas", "-v"] if verbose else []))
    for f in CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OUT, f + ".o")
        objs.append(obj)
        if _stale(obj, src):
            jobs.append(["g++", "-O2", "-fPIC", "-ffp-contract=off", "-std=c++17", "-I", INCLUDE,
                         "-c", src, "-o", obj])
    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for out in ex.map(_compile, jobs):
                if verbose and out:
                    print(out, file=sys.stderr)
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        _compile([nvcc, *ARCH, "-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
