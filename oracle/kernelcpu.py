"""Python wrapper around ``mhs_kernelcpu.c``, the paper's sequential design
(Section 4.2, Algorithms 4-6: explicit I^E / I^V count matrices updated
after each removal, with candidate lists P^E / P^V).

TEST AND BASELINE INFRASTRUCTURE ONLY: the tests and the benchmark's CPU
baseline call it; the product path never does.  It shares no code with the
pairwise oracle (``mhs_oracle.c``) or with the CUDA library, which makes it a
third, independent implementation for the parity tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhs_kernelcpu.c")
_BUILD = os.path.join(_HERE, "_build")
_OUT = os.path.join(_BUILD, "libmhs_kernelcpu.so")
_LOCK = threading.Lock()
_LIB = None

# Dense count matrices larger than this are refused (m^2 + n^2 entries).
DEFAULT_MAX_BYTES = 8 << 30


def build(force: bool = False) -> str:
    """Compile with gcc, with OpenMP when the compiler has it."""
    with _LOCK:
        if (not force and os.path.exists(_OUT)
                and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
            return _OUT
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                           stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        i32p, u8p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8)
        lib.mhs_kernelcpu.argtypes = [i32, i32, i32p, i32p, i32p, i64, i32, u8p, u8p, i32p]
        lib.mhs_kernelcpu.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def reduce(inst, threads: int = 1, max_bytes: int = DEFAULT_MAX_BYTES) -> dict:
    """Kernelize ``inst`` with Algorithm 6; same result dict as the oracle's
    ``reduce``: surviving input vertex / hyperedge ids (ascending), their
    demands, k and the number of DP+MD pass pairs, counting the last one
    that removes nothing."""
    lib = _load()
    n, m = int(inst.n), int(inst.m)
    ptr = np.ascontiguousarray(inst.edge_ptr, dtype=np.int32)
    vtx = np.ascontiguousarray(inst.edge_vtx, dtype=np.int32)
    if vtx.size == 0:
        vtx = np.zeros(1, np.int32)
    dem = np.ascontiguousarray(inst.demand, dtype=np.int32)
    if dem.size == 0:
        dem = np.zeros(1, np.int32)
    av = np.zeros(max(n, 1), np.uint8)
    ae = np.zeros(max(m, 1), np.uint8)
    rounds = ctypes.c_int32(0)
    i32, u8 = ctypes.c_int32, ctypes.c_uint8
    rc = lib.mhs_kernelcpu(n, m, _p(ptr, i32), _p(vtx, i32), _p(dem, i32), int(max_bytes),
                           int(threads), _p(av, u8), _p(ae, u8), ctypes.byref(rounds))
    if rc == -2:
        raise MemoryError(f"dense count matrices for n={n}, m={m} exceed {max_bytes} bytes")
    if rc != 0:
        raise MemoryError("allocation failed")
    edges = np.nonzero(ae[:m])[0].astype(np.int32)
    return {
        "vertices": np.nonzero(av[:n])[0].astype(np.int32),
        "edges": edges,
        "demands": np.asarray(inst.demand, dtype=np.int32)[edges],
        "k": int(inst.k),
        "rounds": int(rounds.value),
    }


def matrix_bytes(n: int, m: int, wide: bool = False) -> int:
    return (4 if wide else 2) * (int(m) * int(m) + int(n) * int(n))
