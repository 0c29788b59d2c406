"""Every tile shape of the tcgen05 contraction gives the oracle's result.

The shape (128 x 256 or 128 x 128 tiles, row blocks per L2 group, half
stages on or off) changes only speed; the autotuner picks one per size
class.  Each shape is run on instances that span several tiles, ragged
edges, both hyperedge rules, rule FE, large counts (the FP32 epilogue) and
a batch, and compared bit-exact with the oracle.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_06042_gb300 import instances as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SHAPES = [dict(tile_n=tn, group_rows=g, half_stages=h)
          for tn in (128, 256) for g in (1, 16) for h in (True, False)]


@pytest.fixture(scope="module")
def mhs():
    from paper_2109_06042_gb300 import build
    build.build()
    from paper_2109_06042_gb300 import mhs as M
    return M


def _same(gpu, ref, ctx=""):
    for key in ("vertices", "edges", "demands"):
        assert gpu[key].tolist() == ref[key].tolist(), f"{key} differ {ctx}"
    assert gpu["k"] == ref["k"], ctx
    assert gpu["rounds"] == ref["rounds"], f"rounds {gpu['rounds']} != {ref['rounds']} {ctx}"


def _cases():
    return [I.config_uniform(3), I.config_uniform(4),
            I.uniform_random(700, 1500, 1, 8, 4, 70, 91_000),
            I.uniform_random(257, 640, 2, 6, 3, 30, 91_001),
            I.config_powerlaw(2, n=3000, m=6000),
            I.config_interval(2, n=3000, m=6000)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"n{s['tile_n']}_g{s['group_rows']}_h{int(s['half_stages'])}")
def test_every_shape_matches_the_oracle(mhs, shape):
    for inst in _cases():
        ref = O.reduce(inst)
        with mhs.Instance.load(inst, contraction="fp8", tiles=shape) as h:
            cfg = h.tile_config()
            assert cfg["tile_n"] == shape["tile_n"] and cfg["group_rows"] == shape["group_rows"]
            assert cfg["half_stages"] == shape["half_stages"] and not cfg["from_table"]
            h.kernelize()
            _same(h.result(), ref, f"{inst.name} {shape}")


@pytest.mark.parametrize("tile_n", [128, 256])
def test_shapes_with_variants_and_dense(mhs, tile_n):
    """SE and FE epilogues, and the dense formulation, at both widths."""
    tiles = dict(tile_n=tile_n)
    for inst in (I.uniform_random(700, 1500, 1, 8, 4, 70, 91_002), I.config_powerlaw(5, n=2000, m=4000)):
        for rule, fe in (("dp", False), ("se", False), ("dp", True), ("se", True)):
            got = mhs.kernelize(inst, contraction="fp8", rule=rule, full_edges=fe, tiles=tiles)
            ref = O.reduce_variant(inst, rule, fe)
            _same(got, ref, f"{inst.name} {rule} fe={fe} tile_n={tile_n}")
        got = mhs.kernelize(inst, contraction="fp8", sparsity="dense", tiles=tiles)
        _same(got, O.reduce(inst), f"{inst.name} dense tile_n={tile_n}")


@pytest.mark.parametrize("tile_n", [128, 256])
def test_large_counts_take_the_fp32_epilogue(mhs, tile_n):
    """Hyperedges {0, 1, a, b} over all pairs a < b: vertices 0 and 1 have
    degree m > 1024, so no tile of the MD pass is drained as FP16 and the
    FP32 tests decide; the result is the closed form checked by the oracle."""
    nb = 60
    pairs = [(a, b) for a in range(2, nb + 2) for b in range(a + 1, nb + 2)]
    edges = [[0, 1, a, b] for a, b in pairs]
    inst = I.from_edges(nb + 2, edges, [1] * len(edges))
    assert len(edges) > 1024
    _same(mhs.kernelize(inst, contraction="fp8", tiles=dict(tile_n=tile_n)), O.reduce(inst),
          f"tile_n={tile_n}")


@pytest.mark.parametrize("tile_n", [128, 256])
def test_batch_at_both_widths(mhs, tile_n):
    insts = [I.config_batch_one(4000 + s) for s in range(12)] + [
        I.from_edges(0, [], []), I.from_edges(4, [], []), I.config_uniform(9)]
    with mhs.Instance.load_batch(insts, contraction="fp8", tiles=dict(tile_n=tile_n)) as h:
        h.kernelize()
        for b, inst in enumerate(insts):
            _same(h.result(b), O.reduce(inst), f"instance {b} tile_n={tile_n}")


def test_invalid_tile_options_rejected(mhs):
    inst = I.config_uniform(0)
    for bad in (dict(tile_n=64), dict(tile_n=512), dict(group_rows=-1), dict(group_rows=5000)):
        with pytest.raises(mhs.MhsError) as ei:
            mhs.Instance.load(inst, contraction="fp8", tiles=bad)
        assert ei.value.status == mhs.MHS_EINVAL
    o = mhs.make_options("fp8")
    o.tile_m = 64
    import ctypes
    h = ctypes.c_void_p()
    ptr = np.ascontiguousarray(inst.edge_ptr, np.int32)
    vtx = np.ascontiguousarray(inst.edge_vtx, np.int32)
    dem = np.ascontiguousarray(inst.demand, np.int32)
    st = mhs.lib().mhs_load(inst.n, inst.m, mhs._p32(ptr), mhs._p32(vtx), mhs._p32(dem), inst.k,
                            ctypes.byref(o), None, ctypes.byref(h))
    assert st == mhs.MHS_EINVAL


def test_table_choice_is_used(tmp_path):
    """A tile table (MHS_TILE_TABLE) sets the shape of loads that leave it
    to the autotuner, by size class; explicit options still win.  The table
    is read once per process, so the check runs in a child process."""
    table = tmp_path / "tiles.txt"
    table.write_text("# kind log2rows tile_n group_rows half_stages\n"
                     "single 8 128 4 2\n"
                     "single 15 256 32 1\n"
                     "batch 10 128 8 1\n"
                     "garbage line\n")
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from oracle import oracle as O\n"
        "from paper_2109_06042_gb300 import instances as I, mhs\n"
        "u = I.config_uniform(1)\n"
        "with mhs.Instance.load(u, contraction='fp8') as h:\n"
        "    c = h.tile_config()\n"
        "    assert c == dict(tile_n=128, group_rows=4, half_stages=False, from_table=True), c\n"
        "    h.kernelize(); r = h.result()\n"
        "ref = O.reduce(u)\n"
        "assert r['vertices'].tolist() == ref['vertices'].tolist() and r['rounds'] == ref['rounds']\n"
        "with mhs.Instance.load(u, contraction='fp8', tiles=dict(tile_n=256)) as h:\n"
        "    c = h.tile_config()\n"
        "    assert c['tile_n'] == 256 and c['group_rows'] == 4, c\n"
        "b = [I.config_batch_one(4000 + s) for s in range(4)]\n"
        "with mhs.Instance.load_batch(b, contraction='fp8') as h:\n"
        "    c = h.tile_config()\n"
        "    assert c == dict(tile_n=128, group_rows=8, half_stages=True, from_table=True), c\n"
        "    h.kernelize()\n"
        "    for i, inst in enumerate(b):\n"
        "        assert h.result(i)['edges'].tolist() == O.reduce(inst)['edges'].tolist()\n"
        "print('table ok')\n" % ROOT)
    env = dict(os.environ, MHS_TILE_TABLE=str(table))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0 and "table ok" in out.stdout, out.stderr[-3000:]
