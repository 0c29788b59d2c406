"""Python wrapper around the C oracle (``mhs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline are the only callers.  The product path (the CUDA library and its
binding) never imports this module.

``reduce()`` runs Algorithm 3 (DP passes of Algorithm 1 alternating with MD
passes of Algorithm 2, Section 4.1) to a fixpoint and returns the surviving
input ids, their demands, k and the round count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

# Planted mistakes, compiled into separate libraries by the mutation tests.
MUTANTS = (
    "DP_TRANSPOSED",
    "DP_DROP_FI",
    "DP_TIEBREAK_HIGH",
    "DP_NO_TIEBREAK",
    "MD_STRICT_ONLY",
    "MD_TIEBREAK_HIGH",
    "MD_MAXF_ALL_EDGES",
    "MD_STRICT_GT",
    "MD_KEEP_ISOLATED",
    "SEQUENTIAL_MD_BEFORE_DP",
    "SE_IGNORE_DEMAND",
    "SE_DEMAND_REVERSED",
    "FE_K_UNCHANGED",
    "FE_SKIP_DECREMENT",
    "FE_KEEP_ZERO_DEMAND",
    "FE_NO_ALTERNATION",
)


def lib_path(mutant: str | None = None) -> str:
    name = "libmhs_oracle.so" if mutant is None else f"libmhs_oracle_{mutant}.so"
    return os.path.join(_BUILD, name)


def build(mutant: str | None = None, force: bool = False) -> str:
    """Compile the oracle (or one planted-mistake variant) with gcc."""
    out = lib_path(mutant)
    with _LOCK:
        if (not force and os.path.exists(out)
                and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
            return out
        os.makedirs(_BUILD, exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC]
        if mutant is not None:
            cmd.insert(1, f"-DORACLE_MUTANT_{mutant}")
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _load(mutant: str | None = None):
    key = mutant or ""
    if key in _LIBS:
        return _LIBS[key]
    lib = ctypes.CDLL(build(mutant))
    i32, u8p, i32p = ctypes.c_int32, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int32)
    lib.mhs_oracle_reduce.argtypes = [i32, i32, i32p, i32p, i32p, i32, i32, u8p, u8p,
                                      i32p, i32p, i32p, i32]
    lib.mhs_oracle_reduce.restype = ctypes.c_int
    lib.mhs_oracle_dp_pass.argtypes = [i32, i32, i32p, i32p, i32p, i32, u8p, u8p, u8p]
    lib.mhs_oracle_dp_pass.restype = ctypes.c_int
    lib.mhs_oracle_md_pass.argtypes = [i32, i32, i32p, i32p, i32p, i32, u8p, u8p, u8p, i32p, i32p]
    lib.mhs_oracle_md_pass.restype = ctypes.c_int
    i64, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)
    lib.mhs_oracle_reduce_ext.argtypes = [i32, i32, i32p, i32p, i32p, i64, i32, i32, i32, i32,
                                          u8p, u8p, i32p, u8p, i64p, i32p, i32p, i32p]
    lib.mhs_oracle_reduce_ext.restype = ctypes.c_int
    lib.mhs_oracle_supersedes.argtypes = [i32, i32, i32p, i32p, i32p, u8p, i32, i32]
    lib.mhs_oracle_supersedes.restype = ctypes.c_int
    lib.mhs_oracle_dominates.argtypes = [i32, i32, i32p, i32p, u8p, i32, i32]
    lib.mhs_oracle_dominates.restype = ctypes.c_int
    _LIBS[key] = lib
    return lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _Arrays:
    """Keeps contiguous copies of an instance's arrays alive for a call."""

    def __init__(self, inst):
        self.n, self.m = int(inst.n), int(inst.m)
        self.ptr = np.ascontiguousarray(inst.edge_ptr, dtype=np.int32)
        vtx = np.ascontiguousarray(inst.edge_vtx, dtype=np.int32)
        self.vtx = vtx if vtx.size else np.zeros(1, np.int32)
        self.dem = np.ascontiguousarray(inst.demand, dtype=np.int32)
        if self.dem.size == 0:
            self.dem = np.zeros(1, np.int32)

    def args(self):
        i32 = ctypes.c_int32
        return (self.n, self.m, _p(self.ptr, i32), _p(self.vtx, i32), _p(self.dem, i32))


def _alive(size, given):
    if given is None:
        return np.ones(max(size, 1), dtype=np.uint8)
    a = np.zeros(max(size, 1), dtype=np.uint8)
    a[:size] = np.asarray(given, dtype=np.uint8)[:size]
    return a


def reduce_state(inst, alive_v=None, alive_e=None, max_rounds: int = 0, prune: bool = True,
                 mutant: str | None = None, trace_cap: int = 0):
    """Run Algorithm 3 from a given alive state.

    Returns (alive_v, alive_e, rounds, changed, trace) with alive masks over
    the input ids and, if ``trace_cap`` > 0, an int32[rounds, 4] array of
    [edges deleted by DP, vertices deleted by MD, alive edges, alive vertices].
    """
    lib = _load(mutant)
    arr = _Arrays(inst)
    av = _alive(arr.n, alive_v)
    ae = _alive(arr.m, alive_e)
    rounds = ctypes.c_int32(0)
    changed = ctypes.c_int32(0)
    trace = np.zeros((max(trace_cap, 1), 4), dtype=np.int32)
    rc = lib.mhs_oracle_reduce(*arr.args(), int(max_rounds), int(bool(prune)),
                               _p(av, ctypes.c_uint8), _p(ae, ctypes.c_uint8),
                               ctypes.byref(rounds), ctypes.byref(changed),
                               _p(trace, ctypes.c_int32), int(trace_cap))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    r = int(rounds.value)
    return (av[:arr.n].astype(bool), ae[:arr.m].astype(bool), r, bool(changed.value),
            trace[:min(r, trace_cap)] if trace_cap > 0 else None)


def reduce(inst, prune: bool = True, max_rounds: int = 0, mutant: str | None = None) -> dict:
    """Kernelize ``inst`` (Algorithm 3 to a fixpoint, or ``max_rounds`` rounds).

    Returns a dict with the surviving input vertex ids and hyperedge ids
    (ascending), the surviving hyperedges' demands (unchanged inputs), k
    (unchanged) and the number of rounds executed, counting the final round
    that changes nothing.
    """
    av, ae, rounds, changed, _ = reduce_state(inst, max_rounds=max_rounds, prune=prune,
                                              mutant=mutant)
    edges = np.nonzero(ae)[0].astype(np.int32)
    return {
        "vertices": np.nonzero(av)[0].astype(np.int32),
        "edges": edges,
        "demands": np.asarray(inst.demand, dtype=np.int32)[edges],
        "k": int(inst.k),
        "rounds": rounds,
        "changed": changed,
    }


RULES = {"dp": 0, "se": 1}


def reduce_variant(inst, rule: str = "dp", full_edges: bool = False, prune: bool = True,
                   max_rounds: int = 0, mutant: str | None = None) -> dict:
    """The reduction variants of the experiments (Section 5.1): Algorithm 3
    with DP ("dp") or the superedge rule SE ("se") as its hyperedge pass,
    and with ``full_edges`` alternated with exhaustive FE (KernelGPU-FE).

    Returns the dict of ``reduce`` with the CURRENT demands of the surviving
    hyperedges (FE lowers them), the current k, ``forced`` (input ids of the
    vertices FE put into the solution, ascending) and ``fe_passes``.
    """
    lib = _load(mutant)
    arr = _Arrays(inst)
    av = _alive(arr.n, None)
    ae = _alive(arr.m, None)
    fo = np.zeros(max(arr.m, 1), dtype=np.int32)
    forced = np.zeros(max(arr.n, 1), dtype=np.uint8)
    k_out = ctypes.c_int64(0)
    rounds, passes, changed = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    rc = lib.mhs_oracle_reduce_ext(*arr.args(), int(inst.k), RULES[rule], int(bool(full_edges)),
                                   int(max_rounds), int(bool(prune)), _p(av, ctypes.c_uint8),
                                   _p(ae, ctypes.c_uint8), _p(fo, ctypes.c_int32),
                                   _p(forced, ctypes.c_uint8), ctypes.byref(k_out),
                                   ctypes.byref(rounds), ctypes.byref(passes),
                                   ctypes.byref(changed))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    edges = np.nonzero(ae[:arr.m])[0].astype(np.int32)
    return {
        "vertices": np.nonzero(av[:arr.n])[0].astype(np.int32),
        "edges": edges,
        "demands": fo[:arr.m][edges].astype(np.int32),
        "k": int(k_out.value),
        "rounds": int(rounds.value),
        "fe_passes": int(passes.value),
        "forced": np.nonzero(forced[:arr.n])[0].astype(np.int32),
        "changed": bool(changed.value),
    }


def dp_pass(inst, alive_v, alive_e, prune: bool = True, mutant: str | None = None):
    """One pass of Algorithm 1; returns the bool mask of deleted hyperedges."""
    lib = _load(mutant)
    arr = _Arrays(inst)
    av, ae = _alive(arr.n, alive_v), _alive(arr.m, alive_e)
    de = np.zeros(max(arr.m, 1), dtype=np.uint8)
    rc = lib.mhs_oracle_dp_pass(*arr.args(), int(bool(prune)), _p(av, ctypes.c_uint8),
                                _p(ae, ctypes.c_uint8), _p(de, ctypes.c_uint8))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return de[:arr.m].astype(bool)


def md_pass(inst, alive_v, alive_e, prune: bool = True, mutant: str | None = None):
    """One pass of Algorithm 2; returns (deleted-vertex mask, C_j, maxf_j)."""
    lib = _load(mutant)
    arr = _Arrays(inst)
    av, ae = _alive(arr.n, alive_v), _alive(arr.m, alive_e)
    dv = np.zeros(max(arr.n, 1), dtype=np.uint8)
    cnt = np.zeros(max(arr.n, 1), dtype=np.int32)
    mxf = np.zeros(max(arr.n, 1), dtype=np.int32)
    rc = lib.mhs_oracle_md_pass(*arr.args(), int(bool(prune)), _p(av, ctypes.c_uint8),
                                _p(ae, ctypes.c_uint8), _p(dv, ctypes.c_uint8),
                                _p(cnt, ctypes.c_int32), _p(mxf, ctypes.c_int32))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return dv[:arr.n].astype(bool), cnt[:arr.n], mxf[:arr.n]


def supersedes(inst, alive_v, i: int, j: int) -> bool:
    lib = _load()
    arr = _Arrays(inst)
    av = _alive(arr.n, alive_v)
    return bool(lib.mhs_oracle_supersedes(*arr.args(), _p(av, ctypes.c_uint8), int(i), int(j)))


def dominates(inst, alive_e, i: int, j: int) -> bool:
    lib = _load()
    arr = _Arrays(inst)
    ae = _alive(arr.m, alive_e)
    return bool(lib.mhs_oracle_dominates(arr.n, arr.m, _p(arr.ptr, ctypes.c_int32),
                                         _p(arr.vtx, ctypes.c_int32), _p(ae, ctypes.c_uint8),
                                         int(i), int(j)))
