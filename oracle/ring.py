"""ctypes front end of oracle/ring_ref.c (definitional NTT and schoolbook
products).  TEST INFRASTRUCTURE ONLY (see oracle/__init__).

``build()`` compiles ring_ref.c with the host C compiler into
oracle/_build/liboracle.so (plain C, OpenMP over output indices).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ring_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.oracle_ntt_eval.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                      u32p, ctypes.c_uint32, u64p]
        L.oracle_ntt.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u64p]
        L.oracle_intt.argtypes = [u64p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u64p]
        L.oracle_negacyclic_mul_small.argtypes = [u64p, i64p, ctypes.c_uint32, ctypes.c_uint64, u64p]
        L.oracle_negacyclic_mul.argtypes = [u64p, u64p, ctypes.c_uint32, ctypes.c_uint64, u64p]
        L.oracle_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def ntt(a, q, psi):
    """Forward negacyclic NTT of a residue vector (definition, O(N^2))."""
    a = _u64(a)
    out = np.empty_like(a)
    lib().oracle_ntt(_ptr(a, ctypes.c_uint64), a.shape[0], q, psi, _ptr(out, ctypes.c_uint64))
    return out


def ntt_eval(a, q, psi, idx):
    """Selected outputs ahat[idx] of the forward NTT (O(N) each)."""
    a = _u64(a)
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    out = np.empty(idx.shape[0], dtype=np.uint64)
    lib().oracle_ntt_eval(_ptr(a, ctypes.c_uint64), a.shape[0], q, psi,
                          _ptr(idx, ctypes.c_uint32), idx.shape[0], _ptr(out, ctypes.c_uint64))
    return out


def intt(ahat, q, psi):
    """Inverse negacyclic NTT (definition, O(N^2))."""
    a = _u64(ahat)
    out = np.empty_like(a)
    lib().oracle_intt(_ptr(a, ctypes.c_uint64), a.shape[0], q, psi, _ptr(out, ctypes.c_uint64))
    return out


def negacyclic_mul_small(a, b, q):
    """a (residues mod q) times b (small signed integers) in Z_q[X]/(X^N+1)."""
    a = _u64(a)
    b = np.ascontiguousarray(b, dtype=np.int64)
    out = np.empty_like(a)
    lib().oracle_negacyclic_mul_small(_ptr(a, ctypes.c_uint64), _ptr(b, ctypes.c_int64),
                                      a.shape[0], q, _ptr(out, ctypes.c_uint64))
    return out


def negacyclic_mul(a, b, q):
    """a times b, both residues mod q, in Z_q[X]/(X^N+1)."""
    a = _u64(a)
    b = _u64(b)
    out = np.empty_like(a)
    lib().oracle_negacyclic_mul(_ptr(a, ctypes.c_uint64), _ptr(b, ctypes.c_uint64),
                                a.shape[0], q, _ptr(out, ctypes.c_uint64))
    return out


def threads() -> int:
    return int(lib().oracle_threads())


def to_residues(v, q):
    """Signed integers (int64 array) -> residues in [0, q) (uint64)."""
    return np.mod(np.asarray(v, dtype=np.int64), np.int64(q)).astype(np.uint64)
