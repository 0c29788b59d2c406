"""Python binding of the C ABI in ``include/mhs.h`` (ctypes; marshalling only).

Every step of the reduction runs in ``libmhs.so``; this module only converts
arguments.  If the library has not been built, importing works but every
call raises ``MhsError`` -- there is no fallback implementation.

Example::

    from paper_2109_06042_gb300 import mhs, instances
    inst = instances.config_uniform(seed=0)
    res = mhs.kernelize(inst)            # dict of surviving ids, demands, k, rounds
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmhs.so")

CONTRACTIONS = {"auto": 0, "fp8": 1, "popcount": 2}

MHS_OK, MHS_EINVAL, MHS_ENOMEM, MHS_ECUDA, MHS_EAGAIN, MHS_ETIMEDOUT, MHS_EBUSY, MHS_EDEVICE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EAGAIN", "ETIMEDOUT", "EBUSY", "EDEVICE"]


class MhsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


LAYOUTS = {"auto": 0, "input": 1, "sorted": 2, "degree": 3}
SPARSITY = {"auto": 0, "skip": 1, "dense": 2}
RULES = {"dp": 0, "se": 1}


class Options(ctypes.Structure):
    _fields_ = [("contraction", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("use_graphs", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("sparsity", ctypes.c_int32), ("edge_rule", ctypes.c_int32),
                ("full_edges", ctypes.c_int32), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("group_rows", ctypes.c_int32),
                ("half_stages", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class RoundStats(ctypes.Structure):
    _fields_ = [("n_alive", ctypes.c_int32), ("m_alive", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("changed", ctypes.c_int32),
                ("dp_deleted", ctypes.c_int32), ("md_deleted", ctypes.c_int32),
                ("active", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("contraction", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("sparsity", ctypes.c_int32),
                ("small_items", ctypes.c_int32), ("edge_rule", ctypes.c_int32),
                ("full_edges", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("rounds", ctypes.c_int64),
                ("pending", ctypes.c_int32), ("active", ctypes.c_int32),
                ("bytes_in_use", ctypes.c_int64), ("peak_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


_lib = None

_i32, _i64, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
_P32 = ctypes.POINTER(ctypes.c_int32)
_P64 = ctypes.POINTER(ctypes.c_int64)
_PU8 = ctypes.POINTER(ctypes.c_uint8)

_SIGS = {
    "mhs_default_options": (_i32, [ctypes.POINTER(Options)]),
    "mhs_load": (_i32, [_i32, _i32, _P32, _P32, _P32, _i64, ctypes.POINTER(Options), _vp,
                        ctypes.POINTER(_vp)]),
    "mhs_load_device": (_i32, [_i32, _i32, _vp, _vp, _vp, _i64, ctypes.POINTER(Options), _vp,
                               ctypes.POINTER(_vp)]),
    "mhs_load_batch": (_i32, [_i32, _P32, _P32, _P64, _P32, _P32, _P64, ctypes.POINTER(Options),
                              _vp, ctypes.POINTER(_vp)]),
    "mhs_load_batch_device": (_i32, [_i32, _P32, _P32, _vp, _vp, _vp, _P64,
                                     ctypes.POINTER(Options), _vp, ctypes.POINTER(_vp)]),
    "mhs_count": (_i32, [_vp]),
    "mhs_reduce_round": (_i32, [_vp, ctypes.POINTER(RoundStats)]),
    "mhs_kernelize": (_i32, [_vp, ctypes.POINTER(RoundStats)]),
    "mhs_pass_begin": (_i32, [_vp, _i32]),
    "mhs_pass_contract": (_i32, [_vp, _i32, _i32, _i32]),
    "mhs_pass_partial": (_i32, [_vp, _i32, _vp, _P64]),
    "mhs_pass_merge": (_i32, [_vp, _i32, _vp]),
    "mhs_pass_end": (_i32, [_vp, _i32, ctypes.POINTER(RoundStats)]),
    "mhs_result_at": (_i32, [_vp, _i32, _P32, _i32, _P32, _P32, _P32, _i32, _P32, _P64, _P32]),
    "mhs_result": (_i32, [_vp, _P32, _i32, _P32, _P32, _P32, _i32, _P32, _P64, _P32]),
    "mhs_forced_at": (_i32, [_vp, _i32, _P32, _i32, _P32, _P32]),
    "mhs_result_device": (_i32, [_vp, _i32, _vp, _vp]),
    "mhs_result_batch_device": (_i32, [_vp, _vp, _vp]),
    "mhs_trace_at": (_i32, [_vp, _i32, _P32, _i32, _P32]),
    "mhs_export": (_i32, [_vp, _i32, _P32, _i32, _P32, _i64, _P32, _P32, _P32, _P64]),
    "mhs_set_timing": (_i32, [_vp, _i32]),
    "mhs_work_stats": (_i32, [_vp, _P64, _P64]),
    "mhs_last_timing": (_i32, [_vp, ctypes.POINTER(ctypes.c_float)]),
    "mhs_tile_config": (_i32, [_vp, _P32, _P32, _P32, _P32]),
    "mhs_kernelize_noalloc": (_i32, [_i32, _i32, _vp, _vp, _vp, _i32, _vp, _vp, _P32, _vp,
                                     ctypes.c_char_p, ctypes.c_size_t]),
    "mhs_server_default_options": (_i32, [ctypes.POINTER(ServerOptions)]),
    "mhs_server_create": (_i32, [ctypes.POINTER(ServerOptions), _vp, ctypes.POINTER(_vp)]),
    "mhs_submit": (_i32, [_vp, _i32, _i32, _P32, _P32, _P32, _i64,
                          ctypes.POINTER(ctypes.c_uint64)]),
    "mhs_poll": (_i32, [_vp, ctypes.c_uint64, _i64, _P32, _i32, _P32, _P32, _P32, _i32, _P32,
                        _P64, _P32, _P64]),
    "mhs_server_forced": (_i32, [_vp, ctypes.c_uint64, _P32, _i32, _P32]),
    "mhs_server_pause": (_i32, [_vp, _i32]),
    "mhs_server_get_stats": (_i32, [_vp, ctypes.POINTER(ServerStats)]),
    "mhs_server_destroy": (None, [_vp]),
    "mhs_selftest_bounded_wait": (_i32, [_i64, _P32, _P64]),
    "mhs_free": (None, [_vp]),
    "mhs_last_error": (ctypes.c_char_p, []),
    "mhs_version": (ctypes.c_char_p, []),
}


def exported_names():
    return sorted(_SIGS)


def lib():
    """Load ``libmhs.so`` (raises MhsError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MhsError(MHS_ECUDA, f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2109_06042_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != MHS_OK:
        raise MhsError(status, lib().mhs_last_error().decode(errors="replace"))


def _p32(a):
    return a.ctypes.data_as(_P32)


_DEFAULT_LAYOUT = ["auto"]
_DEFAULT_SPARSITY = ["auto"]
_DEFAULT_VARIANT = ["dp", False]


def set_default_variant(rule: str = "dp", full_edges: bool = False):
    """Reduction variant used by the helpers below when none is given: the
    hyperedge rule ('dp' or 'se') and whether rule FE alternates with it."""
    _DEFAULT_VARIANT[0] = rule
    _DEFAULT_VARIANT[1] = bool(full_edges)


def set_default_sparsity(sparsity: str):
    """Sparsity policy used by the helpers below when none is given ('auto', 'skip', 'dense')."""
    _DEFAULT_SPARSITY[0] = sparsity


def set_default_layout(layout: str):
    """Layout used by the helpers below when none is given ('auto', 'input', 'sorted')."""
    _DEFAULT_LAYOUT[0] = layout


_DEFAULT_TILES = [None]


def set_default_tiles(tiles):
    """Tile shape used by the helpers below when none is given: None (the
    autotuner's choice) or a dict with any of tile_n (128, 256), group_rows
    and half_stages (True / False)."""
    _DEFAULT_TILES[0] = tiles


def make_options(contraction="auto", max_rounds=0, use_graphs=True, layout=None,
                 sparsity=None, rule=None, full_edges=None, tiles=None) -> Options:
    o = Options()
    _check(lib().mhs_default_options(ctypes.byref(o)))
    o.contraction = CONTRACTIONS[contraction] if isinstance(contraction, str) else int(contraction)
    o.max_rounds = int(max_rounds)
    o.use_graphs = int(bool(use_graphs))
    lay = _DEFAULT_LAYOUT[0] if layout is None else layout
    o.layout = LAYOUTS[lay] if isinstance(lay, str) else int(lay)
    sp = _DEFAULT_SPARSITY[0] if sparsity is None else sparsity
    o.sparsity = SPARSITY[sp] if isinstance(sp, str) else int(sp)
    rule = _DEFAULT_VARIANT[0] if rule is None else rule
    full_edges = _DEFAULT_VARIANT[1] if full_edges is None else full_edges
    o.edge_rule = RULES[rule] if isinstance(rule, str) else int(rule)
    o.full_edges = int(bool(full_edges))
    tiles = _DEFAULT_TILES[0] if tiles is None else tiles
    if tiles:
        o.tile_n = int(tiles.get("tile_n", 0))
        o.group_rows = int(tiles.get("group_rows", 0))
        hs = tiles.get("half_stages")
        o.half_stages = 0 if hs is None else (1 if hs else 2)
    return o


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Instance:
    """Handle of one instance (or a batch) loaded on the GPU."""

    def __init__(self, handle, keepalive=None):
        self._h = handle
        self._keep = keepalive

    # ---- loading ----
    @classmethod
    def load(cls, inst, contraction="auto", max_rounds=0, use_graphs=True, stream=None,
             layout=None, sparsity=None, rule=None, full_edges=None, tiles=None):
        """mhs_load from host arrays of an ``instances.Instance``-like object."""
        ptr = np.ascontiguousarray(inst.edge_ptr, dtype=np.int32)
        vtx = np.ascontiguousarray(inst.edge_vtx, dtype=np.int32)
        dem = np.ascontiguousarray(inst.demand, dtype=np.int32)
        if vtx.size == 0:
            vtx = np.zeros(1, np.int32)
        if dem.size == 0:
            dem = np.zeros(1, np.int32)
        opt = make_options(contraction, max_rounds, use_graphs, layout, sparsity, rule, full_edges,
                           tiles)
        h = ctypes.c_void_p()
        _check(lib().mhs_load(int(inst.n), int(inst.m), _p32(ptr), _p32(vtx), _p32(dem),
                              int(inst.k), ctypes.byref(opt), _stream_ptr(stream),
                              ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load_device(cls, n, m, edge_ptr, edge_vtx, demand, k, contraction="auto", max_rounds=0,
                    use_graphs=True, stream=None, layout=None, sparsity=None, rule=None,
                    full_edges=None, tiles=None):
        """mhs_load_device from CUDA tensors (int32, contiguous)."""
        opt = make_options(contraction, max_rounds, use_graphs, layout, sparsity, rule, full_edges,
                           tiles)
        h = ctypes.c_void_p()
        _check(lib().mhs_load_device(int(n), int(m), ctypes.c_void_p(edge_ptr.data_ptr()),
                                     ctypes.c_void_p(edge_vtx.data_ptr()),
                                     ctypes.c_void_p(demand.data_ptr()), int(k),
                                     ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load_batch(cls, insts, contraction="auto", max_rounds=0, use_graphs=True, stream=None,
                   rule=None, full_edges=None, tiles=None):
        """mhs_load_batch from a list of host instances."""
        count = len(insts)
        n = np.array([i.n for i in insts], dtype=np.int32)
        m = np.array([i.m for i in insts], dtype=np.int32)
        k = np.array([i.k for i in insts], dtype=np.int64)
        nnz = np.array([i.nnz for i in insts], dtype=np.int64)
        ptr = np.zeros(int(m.sum()) + 1, dtype=np.int64)
        base = np.concatenate([[0], np.cumsum(nnz)])
        e0 = 0
        for b, i in enumerate(insts):
            ptr[e0:e0 + i.m + 1] = np.asarray(i.edge_ptr, dtype=np.int64) + base[b]
            e0 += i.m
        vtx = np.concatenate([np.asarray(i.edge_vtx, np.int32) for i in insts] + [np.zeros(1, np.int32)])
        dem = np.concatenate([np.asarray(i.demand, np.int32) for i in insts] + [np.zeros(1, np.int32)])
        return cls.load_batch_arrays(count, n, m, ptr, vtx, dem, k, contraction, max_rounds,
                                     use_graphs, stream, rule=rule, full_edges=full_edges,
                                     tiles=tiles)

    @classmethod
    def load_batch_arrays(cls, count, n, m, ptr, vtx, dem, k, contraction="auto", max_rounds=0,
                          use_graphs=True, stream=None, layout=None, sparsity=None, rule=None,
                          full_edges=None, tiles=None):
        opt = make_options(contraction, max_rounds, use_graphs, layout, sparsity, rule, full_edges,
                           tiles)
        h = ctypes.c_void_p()
        _check(lib().mhs_load_batch(int(count), _p32(n), _p32(m), ptr.ctypes.data_as(_P64),
                                    _p32(vtx), _p32(dem), k.ctypes.data_as(_P64),
                                    ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def load_batch_device(cls, n, m, k, edge_ptr, edge_vtx, demand, contraction="auto",
                          max_rounds=0, use_graphs=True, stream=None, layout=None, sparsity=None,
                          rule=None, full_edges=None, tiles=None):
        """mhs_load_batch_device: n, m, k host numpy arrays; edge_ptr (int64),
        edge_vtx, demand (int32) CUDA tensors over the concatenated instances."""
        n = np.ascontiguousarray(n, dtype=np.int32)
        m = np.ascontiguousarray(m, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int64)
        opt = make_options(contraction, max_rounds, use_graphs, layout, sparsity, rule, full_edges,
                           tiles)
        h = ctypes.c_void_p()
        _check(lib().mhs_load_batch_device(int(n.size), _p32(n), _p32(m),
                                           ctypes.c_void_p(edge_ptr.data_ptr()),
                                           ctypes.c_void_p(edge_vtx.data_ptr()),
                                           ctypes.c_void_p(demand.data_ptr()),
                                           k.ctypes.data_as(_P64), ctypes.byref(opt),
                                           _stream_ptr(stream), ctypes.byref(h)))
        return cls(h)

    # ---- running ----
    def reduce_round(self) -> dict:
        st = RoundStats()
        _check(lib().mhs_reduce_round(self._h, ctypes.byref(st)))
        return st.as_dict()

    def kernelize(self) -> dict:
        st = RoundStats()
        _check(lib().mhs_kernelize(self._h, ctypes.byref(st)))
        return st.as_dict()

    # ---- sharded passes (see paper_2109_06042_gb300/shard.py) ----
    def pass_begin(self, phase: int):
        _check(lib().mhs_pass_begin(self._h, int(phase)))

    def pass_contract(self, phase: int, shard: int, nshards: int):
        _check(lib().mhs_pass_contract(self._h, int(phase), int(shard), int(nshards)))

    def pass_elems(self, phase: int) -> int:
        """Elements of the phase's partial buffer (m flags or n counts)."""
        e = ctypes.c_int64()
        _check(lib().mhs_pass_partial(self._h, int(phase), None, ctypes.byref(e)))
        return int(e.value)

    def pass_partial(self, phase: int, out):
        """Copy the partial flags (uint8) / counts (int32) into a CUDA tensor."""
        e = ctypes.c_int64()
        _check(lib().mhs_pass_partial(self._h, int(phase), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.byref(e)))
        return int(e.value)

    def pass_merge(self, phase: int, buf):
        _check(lib().mhs_pass_merge(self._h, int(phase), ctypes.c_void_p(buf.data_ptr())))

    def pass_end(self, phase: int) -> dict:
        st = RoundStats()
        _check(lib().mhs_pass_end(self._h, int(phase), ctypes.byref(st)))
        return st.as_dict()

    def set_timing(self, enable=True):
        _check(lib().mhs_set_timing(self._h, int(bool(enable))))

    def last_timing(self):
        a = (ctypes.c_float * 4)()
        _check(lib().mhs_last_timing(self._h, a))
        return {"dp_ms": a[0], "md_ms": a[1], "other_ms": a[2], "total_ms": a[3]}

    def tile_config(self) -> dict:
        """The tcgen05 tile shape of this load (options, table or defaults)."""
        v = [ctypes.c_int32() for _ in range(4)]
        _check(lib().mhs_tile_config(self._h, *[ctypes.byref(x) for x in v]))
        return {"tile_n": v[0].value, "group_rows": v[1].value,
                "half_stages": bool(v[2].value), "from_table": bool(v[3].value)}

    def work_stats(self):
        """(MMA work in units of 128x128x32 MACs, tiles contracted) since load."""
        kb = ctypes.c_int64()
        tl = ctypes.c_int64()
        _check(lib().mhs_work_stats(self._h, ctypes.byref(kb), ctypes.byref(tl)))
        return int(kb.value), int(tl.value)

    @property
    def count(self) -> int:
        return int(lib().mhs_count(self._h))

    # ---- results ----
    def result(self, index: int = 0) -> dict:
        n = ctypes.c_int32()
        m = ctypes.c_int32()
        k = ctypes.c_int64()
        r = ctypes.c_int32()
        _check(lib().mhs_result_at(self._h, int(index), None, 0, ctypes.byref(n), None, None, 0,
                                   ctypes.byref(m), ctypes.byref(k), ctypes.byref(r)))
        vtx = np.zeros(max(n.value, 1), np.int32)
        edg = np.zeros(max(m.value, 1), np.int32)
        dem = np.zeros(max(m.value, 1), np.int32)
        _check(lib().mhs_result_at(self._h, int(index), _p32(vtx), vtx.size, ctypes.byref(n),
                                   _p32(edg), _p32(dem), edg.size, ctypes.byref(m),
                                   ctypes.byref(k), ctypes.byref(r)))
        return {"vertices": vtx[:n.value], "edges": edg[:m.value], "demands": dem[:m.value],
                "k": int(k.value), "rounds": int(r.value)}

    def forced(self, index: int = 0):
        """(input ids rule FE put into the solution, ascending; FE passes run)."""
        c = ctypes.c_int32()
        p = ctypes.c_int32()
        _check(lib().mhs_forced_at(self._h, int(index), None, 0, ctypes.byref(c), ctypes.byref(p)))
        out = np.zeros(max(c.value, 1), np.int32)
        _check(lib().mhs_forced_at(self._h, int(index), _p32(out), out.size, ctypes.byref(c),
                                   ctypes.byref(p)))
        return out[:c.value], int(p.value)

    def result_device(self, alive_v, alive_e, index: int = 0):
        """Write uint8 alive masks (CUDA tensors) over the input ids."""
        _check(lib().mhs_result_device(self._h, int(index), ctypes.c_void_p(alive_v.data_ptr()),
                                       ctypes.c_void_p(alive_e.data_ptr())))

    def result_batch_device(self, alive_v, alive_e):
        """Concatenated uint8 alive masks of all instances (CUDA tensors)."""
        _check(lib().mhs_result_batch_device(self._h, ctypes.c_void_p(alive_v.data_ptr()),
                                             ctypes.c_void_p(alive_e.data_ptr())))

    def trace(self, index: int = 0):
        """Per-round (hyperedges into DP, vertices into DP, hyperedges after DP)."""
        rows = np.zeros((32, 3), np.int32)
        r = ctypes.c_int32()
        _check(lib().mhs_trace_at(self._h, int(index), _p32(rows), 32, ctypes.byref(r)))
        return rows[:min(r.value, 32)].copy(), int(r.value)

    def export(self, index: int = 0):
        """The current reduced instance as (n, edge_ptr, edge_vtx, demand), renumbered."""
        n = ctypes.c_int32()
        m = ctypes.c_int32()
        nnz = ctypes.c_int64()
        _check(lib().mhs_export(self._h, int(index), None, 0, None, 0, None, ctypes.byref(n),
                                ctypes.byref(m), ctypes.byref(nnz)))
        ptr = np.zeros(m.value + 1, np.int32)
        vtx = np.zeros(max(nnz.value, 1), np.int32)
        dem = np.zeros(max(m.value, 1), np.int32)
        _check(lib().mhs_export(self._h, int(index), _p32(ptr), m.value, _p32(vtx), vtx.size,
                                _p32(dem), ctypes.byref(n), ctypes.byref(m), ctypes.byref(nnz)))
        return int(n.value), ptr, vtx[:nnz.value], dem[:m.value]

    def free(self):
        if self._h:
            lib().mhs_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kernelize(inst, contraction="auto", max_rounds=0, use_graphs=True, layout=None,
              sparsity=None, rule=None, full_edges=None, tiles=None) -> dict:
    """Load, reduce to the fixpoint and return the result of one host instance
    (with ``full_edges`` also 'forced' and 'fe_passes')."""
    with Instance.load(inst, contraction, max_rounds, use_graphs, layout=layout,
                       sparsity=sparsity, rule=rule, full_edges=full_edges, tiles=tiles) as h:
        h.kernelize()
        res = h.result()
        if (_DEFAULT_VARIANT[1] if full_edges is None else full_edges):
            res["forced"], res["fe_passes"] = h.forced()
        return res


class Server:
    """Continuous-batching server (mhs_server_*): submit host instances, poll results."""

    def __init__(self, hbm_budget_bytes=0, max_slots=256, queue_capacity=65536,
                 contraction="auto", stream=None, layout=None, sparsity=None, small_items=0,
                 rule=None, full_edges=None):
        o = ServerOptions()
        _check(lib().mhs_server_default_options(ctypes.byref(o)))
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        o.max_slots = int(max_slots)
        o.queue_capacity = int(queue_capacity)
        o.contraction = CONTRACTIONS[contraction] if isinstance(contraction, str) else int(contraction)
        lay = _DEFAULT_LAYOUT[0] if layout is None else layout
        o.layout = LAYOUTS[lay] if isinstance(lay, str) else int(lay)
        sp = _DEFAULT_SPARSITY[0] if sparsity is None else sparsity
        o.sparsity = SPARSITY[sp] if isinstance(sp, str) else int(sp)
        o.small_items = int(small_items)
        rule = _DEFAULT_VARIANT[0] if rule is None else rule
        full_edges = _DEFAULT_VARIANT[1] if full_edges is None else full_edges
        o.edge_rule = RULES[rule] if isinstance(rule, str) else int(rule)
        o.full_edges = int(bool(full_edges))
        self._fe = bool(full_edges)
        h = ctypes.c_void_p()
        _check(lib().mhs_server_create(ctypes.byref(o), _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def submit(self, inst) -> int:
        ptr = np.ascontiguousarray(inst.edge_ptr, dtype=np.int32)
        vtx = np.ascontiguousarray(inst.edge_vtx, dtype=np.int32)
        dem = np.ascontiguousarray(inst.demand, dtype=np.int32)
        if vtx.size == 0:
            vtx = np.zeros(1, np.int32)
        if dem.size == 0:
            dem = np.zeros(1, np.int32)
        t = ctypes.c_uint64()
        _check(lib().mhs_submit(self._h, int(inst.n), int(inst.m), _p32(ptr), _p32(vtx),
                                _p32(dem), int(inst.k), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket, timeout_us=-1):
        """Result dict (with 'times_ns': queued, in service, total), or None if
        the request is not finished within timeout_us."""
        n = ctypes.c_int32()
        m = ctypes.c_int32()
        k = ctypes.c_int64()
        r = ctypes.c_int32()
        tm = (ctypes.c_int64 * 3)()
        st = lib().mhs_poll(self._h, ctypes.c_uint64(ticket), int(timeout_us), None, 0,
                            ctypes.byref(n), None, None, 0, ctypes.byref(m), ctypes.byref(k),
                            ctypes.byref(r), tm)
        if st == MHS_EAGAIN:
            return None
        _check(st)
        forced = None
        if self._fe:  # before the copying poll releases the result
            c = ctypes.c_int32()
            _check(lib().mhs_server_forced(self._h, ctypes.c_uint64(ticket), None, 0,
                                           ctypes.byref(c)))
            fb = np.zeros(max(c.value, 1), np.int32)
            _check(lib().mhs_server_forced(self._h, ctypes.c_uint64(ticket), _p32(fb), fb.size,
                                           ctypes.byref(c)))
            forced = fb[:c.value]
        vtx = np.zeros(max(n.value, 1), np.int32)
        edg = np.zeros(max(m.value, 1), np.int32)
        dem = np.zeros(max(m.value, 1), np.int32)
        _check(lib().mhs_poll(self._h, ctypes.c_uint64(ticket), 0, _p32(vtx), vtx.size,
                              ctypes.byref(n), _p32(edg), _p32(dem), edg.size, ctypes.byref(m),
                              ctypes.byref(k), ctypes.byref(r), tm))
        res = {"vertices": vtx[:n.value], "edges": edg[:m.value], "demands": dem[:m.value],
               "k": int(k.value), "rounds": int(r.value), "times_ns": [int(x) for x in tm]}
        if forced is not None:
            res["forced"] = forced
        return res

    def pause(self, paused=True):
        _check(lib().mhs_server_pause(self._h, int(bool(paused))))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().mhs_server_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self._h:
            lib().mhs_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernelize_noalloc(n, m, edge_ptr, edge_vtx, demand, nnz, alive_v, alive_e, stream=None):
    """mhs_kernelize_noalloc on CUDA tensors: no memory is allocated by the
    call; alive_v / alive_e (uint8 CUDA tensors) receive the surviving masks.
    Returns the round count."""
    import torch
    n, m, nnz = int(n), int(m), int(nnz)
    dev = torch.cuda.current_device()
    for name, t, dt, need in (("edge_ptr", edge_ptr, torch.int32, m + 1),
                              ("edge_vtx", edge_vtx, torch.int32, nnz),
                              ("demand", demand, torch.int32, m),
                              ("alive_v", alive_v, torch.uint8, n),
                              ("alive_e", alive_e, torch.uint8, m)):
        if not (t.is_cuda and t.device.index == dev):
            raise MhsError(MHS_EINVAL, f"{name} must be a CUDA tensor on device {dev}")
        if t.dtype != dt or not t.is_contiguous():
            raise MhsError(MHS_EINVAL, f"{name} must be a contiguous {dt} tensor")
        if t.numel() < need:
            raise MhsError(MHS_EINVAL, f"{name} holds {t.numel()} elements, needs {need}")
    rounds = ctypes.c_int32(0)
    buf = ctypes.create_string_buffer(256)
    st = lib().mhs_kernelize_noalloc(int(n), int(m), ctypes.c_void_p(edge_ptr.data_ptr()),
                                     ctypes.c_void_p(edge_vtx.data_ptr()),
                                     ctypes.c_void_p(demand.data_ptr()), int(nnz),
                                     ctypes.c_void_p(alive_v.data_ptr()),
                                     ctypes.c_void_p(alive_e.data_ptr()), ctypes.byref(rounds),
                                     _stream_ptr(stream), buf, 256)
    if st != MHS_OK:
        raise MhsError(st, buf.value.decode(errors="replace"))
    return int(rounds.value)


def selftest_bounded_wait(limit_ns=20_000_000):
    """Run the bounded-wait diagnostic; returns (status, waited_ns)."""
    st = ctypes.c_int32()
    w = ctypes.c_int64()
    _check(lib().mhs_selftest_bounded_wait(int(limit_ns), ctypes.byref(st), ctypes.byref(w)))
    return int(st.value), int(w.value)


def version() -> str:
    return lib().mhs_version().decode()
